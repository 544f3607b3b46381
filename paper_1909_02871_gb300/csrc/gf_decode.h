// gf_decode.h -- internal interface of the batched decode.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gf_encode.h"

namespace gf {

constexpr int kMaxDecodeN = 1024;
constexpr int kMaxDecodeR = 4096;

// Device descriptor of one generation's coefficient phase.
struct DecGen {
    const uint8_t *coef;
    const uint8_t *payload;
    uint8_t *out;
    int32_t *rank;
    int32_t *used;
    uint8_t *solved;
    uint8_t *X;      // N x R transform (device scratch)
    uint8_t *grows;  // N x W stored rows in global scratch, or NULL (shared memory)
    unsigned long long len;
    int field, N, R, W;
    size_t x_off, grow_off;  // host-side placement offsets
    int blk;                 // index in DecodeWork::blk, or -1 (decode_coef_kernel)
};

// Blocked coefficient phase (gf_decode_blk.cu) for generations of many
// sources: blocks of kBlkRows arriving rows, row products on the encode.
constexpr int kBlkRows = 64;
constexpr int kBlkMinN = 64;    // sources from which a generation takes the blocked path (measured best)
constexpr int kBlkMaxW = 2048;  // widest rows (N + R, rounded to 16) it takes

struct BlkGen {
    const uint8_t *coef;  // R x N received coding vectors
    uint8_t *S;           // N x W stored rows (reduced), slots 0 .. rank-1 live
    uint8_t *cur;         // kBlkRows x W: the block's rows
    uint8_t *NR;          // kBlkRows x W: the block's new pivot rows
    uint8_t *F;           // kBlkRows x N: block rows in the stored pivot columns
    uint8_t *G;           // N x kBlkRows: stored rows in the new pivot columns
    int *pcol;            // stored row -> pivot column
    int *st;              // [0] rank, [1] rows used
    uint8_t *X;           // N x R transform (output)
    int32_t *rank_out;
    int32_t *used_out;
    uint8_t *solved;
    int field, N, R, W;
    size_t off;           // host-side placement offset in the rows region
};

// Host-side description of a decode batch.
struct DecodeWork {
    std::vector<DecGen> gens;
    std::vector<EncGen> apply;
    std::vector<EncodeBatch> batches;
    size_t x_bytes = 0, grow_bytes = 0, smem = 0;
    DecGen *d_gens = nullptr;
    int n_coef = 0;  // generations of decode_coef_kernel (the others are blocked)
    int coef_threads = 1024;  // its CTA size: 256 when every such generation has at most 64 sources
    // blocked generations and, per step, the batches of their two row products
    std::vector<BlkGen> blk;
    std::vector<std::vector<EncodeBatch>> prod1, prod2;
    BlkGen *d_blk = nullptr;
    int blk_max_w = 0, blk_max_n = 0;
};

bool blk_eligible(int field, int N, int R, int W);
size_t blk_scratch_bytes(const BlkGen &g);
void blk_place(BlkGen &g, char *base);
void blk_products(const std::vector<BlkGen> &gens, int step, std::vector<EncGen> &p1, std::vector<EncGen> &p2);
int launch_blk_init(const BlkGen *d, int n, cudaStream_t s);
int launch_blk_prepare(const BlkGen *d, int n, int step, cudaStream_t s);
int launch_blk_gj(const BlkGen *d, int n, int step, int max_w, cudaStream_t s);
int launch_blk_final(const BlkGen *d, int n, int max_n, cudaStream_t s);

int build_decode(const ::gf_dec_t *gens, int n_gens, DecodeWork &w);
int place_decode(DecodeWork &w, char *dev_x, char *dev_rows);
size_t decode_stage_bytes(const DecodeWork &w);
size_t decode_counters(const DecodeWork &w);  // work counters a staged decode needs
size_t stage_decode(DecodeWork &w, char *host, char *dev_base, size_t off, WorkCounter *counters);
int launch_decode(const DecodeWork &w, cudaStream_t stream);
size_t dec_smem_bytes(int field, int N, int W, bool rows_in_smem);
size_t decode_smem_limit();  // largest dynamic shared memory of a decode CTA on this device

}  // namespace gf
