// gf_encode.h -- internal interface of the batched encode (shared with the
// decode, whose payload phase is an encode with the elimination's transform).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gf_runtime.h"

namespace gf {

// Device-side descriptor of one generation to encode (Eq. 2): out_k =
// sum_i coef[k*coef_ld + i] * src_i for k < n_coded, i < n_src.
struct EncGen {
    const uint8_t *src;
    const uint8_t *coef;
    uint8_t *out;
    unsigned long long len;
    int field, n_src, n_coded, coef_ld;
    int variant;      // tile shape (table path) or 0 (bit-sliced path)
    int col_chunks;   // column tiles
    int k_chunks;     // coded-packet tiles
    int path_hint;    // 0, or the GF_PATH_* this generation takes whatever the batch's path
    int accumulate;   // 1: out ^= the products (the blocked decode's GEMMs), 0: out = the products
};

// Table-path tile shapes: (words per lane, coded packets per warp tile).
struct TableVariant {
    int wpt, kpt;
};
constexpr int kNumTableVariants = 4;
extern const TableVariant kTableVariants[kNumTableVariants];

// One persistent launch over a list of generations.
struct EncodeBatch {
    int kind = 0;  // GF_PATH_TABLE or GF_PATH_BITSLICED
    std::vector<EncGen> gens;
    std::vector<long long> tile_start;  // n_gens + 1 prefix sums
    long long total_tiles = 0;
    bool all_gf256 = true;  // bit-sliced: every generation is GF(256) (specialised kernel)
    bool col_split = false;  // bit-sliced: some item covers only a range of its column tiles
    // device copies (inside a workspace or plan buffer)
    WorkCounter *d_counter = nullptr;
    EncGen *d_gens = nullptr;
    long long *d_tile_start = nullptr;
};

// Fill tile counts and prefix sums for `b.gens` according to b.kind.
void finalize_batch(EncodeBatch &b);

// Bytes needed to upload a batch (gens + tile_start), 256-aligned.
size_t batch_bytes(const EncodeBatch &b);

// Serialise the batch into `host` at byte offset `off` and set the device
// pointers relative to `dev_base` (same offset), return the new offset.
size_t stage_batch(EncodeBatch &b, char *host, char *dev_base, size_t off);

// Enqueue the persistent kernel of a staged batch.
int launch_batch(const EncodeBatch &b, cudaStream_t stream);

// Choose the table-path variant for a generation (autotuner, else heuristic).
int choose_table_variant(int field, int n_src, int n_coded, unsigned long long len);

// Choose the path for a generation under GF_PATH_AUTO.
int choose_path(int field, int n_src, int n_coded, unsigned long long len);

// Whether the bit-sliced (tcgen05) path can run on the current device.
bool bitsliced_available();
// Launch the bounded-wait self-test (gf_selftest_wait).
int launch_wait_selftest(int abort_first, cudaStream_t stream);

// Whether a generation fits the bit-sliced kernel (GF(256), 1 <= N <= 128,
// K >= 1, len >= 1); others of a bit-sliced batch run on the table path.
bool bitsliced_supports(const EncGen &g);

// Split `gens` into per-path batches according to `path` (GF_PATH_*).
// Returns GF_OK, GF_EINVAL or GF_ENOTSUP.
int plan_batches(const std::vector<EncGen> &gens, int path, std::vector<EncodeBatch> &out);

// Validate a public descriptor and convert it.
int convert_gen(const ::gf_gen_t &g, EncGen &e);

// Bit-sliced kernel launch (gf_encode_tc.cu).
int launch_bitsliced(const EncodeBatch &b, cudaStream_t stream);
long long bitsliced_tiles(const EncGen &g, int &col_chunks, int &k_chunks);

}  // namespace gf
