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
};

// Host-side description of a decode batch.
struct DecodeWork {
    std::vector<DecGen> gens;
    std::vector<EncGen> apply;
    std::vector<EncodeBatch> batches;
    size_t x_bytes = 0, grow_bytes = 0, smem = 0;
    DecGen *d_gens = nullptr;
};

int build_decode(const ::gf_dec_t *gens, int n_gens, DecodeWork &w);
int place_decode(DecodeWork &w, char *dev_x, char *dev_rows);
size_t decode_stage_bytes(const DecodeWork &w);
size_t stage_decode(DecodeWork &w, char *host, char *dev_base, size_t off, WorkCounter *counters);
int launch_decode(const DecodeWork &w, cudaStream_t stream);
size_t dec_smem_bytes(int field, int N, int W, bool rows_in_smem);
size_t decode_smem_limit();  // largest dynamic shared memory of a decode CTA on this device

}  // namespace gf
