// gf_plan.cu -- plans (pre-uploaded batches that can be captured in CUDA
// graphs) and the encode autotuner.
//
// Autotuner: a shape bucket is (field, ceil(log2 N), ceil(log2 K),
// ceil(log2 len)).  gf_autotune_encode times every candidate (bit-sliced
// tensor-core path where it applies, every table-path tile shape) on
// synthetic data of that shape and remembers the fastest for the bucket;
// GF_PATH_AUTO consults the table, else a fixed heuristic.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gf_decode.h"
#include "gf_encode.h"
#include "gf_internal.cuh"

struct gf_plan {
    int kind = 0;  // 0 encode, 1 decode
    int device = 0;
    void *dev = nullptr;
    size_t dev_size = 0;
    std::vector<gf::EncodeBatch> batches;
    gf::DecodeWork dec;
};

namespace gf {

// ---------------------------------------------------------------------------
// autotuner state
// ---------------------------------------------------------------------------
struct TuneChoice {
    int path, variant;
};
using TuneKey = std::tuple<int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune;
static thread_local int t_force_variant = -1;
// the candidates and mean times of this thread's last gf_autotune_encode call
static thread_local std::vector<std::pair<TuneChoice, float>> t_last_tune;

static int log2_bucket(unsigned long long v)
{
    int b = 0;
    while ((1ull << b) < v && b < 63) ++b;
    return b;
}

static TuneKey tune_key(int field, int n_src, int n_coded, unsigned long long len)
{
    return TuneKey(field, log2_bucket((unsigned long long)std::max(n_src, 1)),
                   log2_bucket((unsigned long long)std::max(n_coded, 1)), log2_bucket(std::max(len, 1ull)));
}

int choose_table_variant(int field, int n_src, int n_coded, unsigned long long len)
{
    if (t_force_variant >= 0) return t_force_variant;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(tune_key(field, n_src, n_coded, len));
        if (it != g_tune.end() && it->second.path == GF_PATH_TABLE) return it->second.variant;
    }
    (void)n_src;
    if (len <= 160) return 1;             // 128-byte column tiles
    if (len <= 320) return 2;             // 256-byte column tiles
    // 512-byte column tiles: 8 packets per tile (the shape that loads a source ahead) up to 16
    // coded packets -- the tuner's choice on every Fig. 1 point from 512 B up -- else 16
    return n_coded <= 16 ? 3 : 0;
}

int choose_path(int field, int n_src, int n_coded, unsigned long long len)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(tune_key(field, n_src, n_coded, len));
        if (it != g_tune.end()) return it->second.path;
    }
    if (!bitsliced_available() || n_src <= 0 || n_coded <= 0 || len == 0) return GF_PATH_TABLE;
    // Cost model in SM clocks per generation per SM, fitted to the tuner's
    // own timings of 288 shapes on a GB300 (GF(2) and GF(256); N 8..255, K
    // 8..64, len 128..4096, 304-608 generations): a tensor-core pass (128
    // bytes x up to 64 coded packets x up to 64 sources) costs about 2300
    // clocks of handshakes plus about 30 per MMA issued (the bias MMA and one
    // per 8 sources, twice for more than 32 coded packets), and every 32 KB
    // K-block of coefficient matrices built about 300; the table path costs
    // about 50 clocks per source for every 128-byte x 8-packet tile (GF(2),
    // a plain XOR, about 0.55 of that).  With these constants AUTO picks the
    // tuner's choice on 251 of the 288 shapes and is 4 % slower than it on
    // average (the constants fitted to the kernel before its K-block ring and
    // batched MMA issue: 239 shapes, 7 %).
    const int chunks = (n_src + 63) / 64, items = (n_coded + 63) / 64;
    const double tiles = std::ceil((double)len / 128.0);
    double mmas = 0.0, kblocks = 0.0;
    for (int it = 0; it < items; ++it) {
        const int halves = std::min(n_coded - 64 * it, 64) > 32 ? 2 : 1;
        for (int c = 0; c < chunks; ++c) mmas += 1 + halves * ((std::min(n_src - 64 * c, 64) + 7) / 8);
        kblocks += 2.0 * halves * chunks;
    }
    const double bits = tiles * (2300.0 * chunks * items + 30.0 * mmas) + 300.0 * kblocks;
    const double ttiles = tiles * std::ceil(n_coded / 8.0);
    const double table = ttiles * (50.0 * n_src * (field == 1 ? 0.55 : 1.0));
    if (bits < table) return GF_PATH_BITSLICED;
    return GF_PATH_TABLE;
}

// fill a buffer with a cheap hash (synthetic tuning data); values < q when
// q != 0
__global__ void fill_kernel(uint8_t *p, size_t n, uint32_t seed, uint32_t q)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 0x9E3779B9u ^ seed;
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        p[i] = (uint8_t)(q ? (x % q) : x);
    }
}

}  // namespace gf

using namespace gf;

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
static int plan_alloc(gf_plan *p, size_t bytes)
{
    p->device = current_device();
    if (cudaMalloc(&p->dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->dev = nullptr;
        return GF_ENOMEM;
    }
    p->dev_size = bytes;
    return cuda_status(cudaMemset(p->dev, 0, kCounterBytes));
}

extern "C" int gf_encode_plan_create(const gf_gen_t *gens, int n_gens, int path, gf_plan_t **plan)
{
    if (!plan || n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    if (path < GF_PATH_AUTO || path > GF_PATH_BITSLICED) return GF_EINVAL;
    *plan = nullptr;
    std::vector<EncGen> eg(n_gens);
    for (int i = 0; i < n_gens; ++i) {
        int st = convert_gen(gens[i], eg[i]);
        if (st != GF_OK) return st;
    }
    gf_plan *p = new gf_plan();
    p->kind = 0;
    int st = plan_batches(eg, path, p->batches);
    if (st != GF_OK) {
        delete p;
        return st;
    }
    size_t bytes = 0;
    for (auto &b : p->batches) bytes += batch_bytes(b);
    st = plan_alloc(p, kCounterBytes + bytes);
    if (st != GF_OK) {
        delete p;
        return st;
    }
    std::vector<char> host(bytes + 16);
    size_t off = 0;
    for (size_t i = 0; i < p->batches.size(); ++i) {
        p->batches[i].d_counter = reinterpret_cast<WorkCounter *>((char *)p->dev + 16 * i);
        off = stage_batch(p->batches[i], host.data(), (char *)p->dev + kCounterBytes, off);
    }
    if (off && cudaMemcpy((char *)p->dev + kCounterBytes, host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
        gf_plan_destroy(p);
        return GF_ECUDA;
    }
    *plan = p;
    return GF_OK;
}

// A recode plan is the encode plan of its payload and coding-vector encodes
// (gf_recode_batched's decomposition).
extern "C" int gf_recode_plan_create(const gf_recode_t *gens, int n_gens, gf_plan_t **plan)
{
    if (!plan || n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    *plan = nullptr;
    std::vector<gf_gen_t> enc;
    enc.reserve(2 * (size_t)n_gens);
    for (int i = 0; i < n_gens; ++i) {
        const gf_recode_t &r = gens[i];
        if (r.n_src < 0 || r.n_in < 0 || r.n_out < 0) return GF_EINVAL;
        enc.push_back(gf_gen_t{r.field, r.n_in, r.n_out, 0, r.len, r.payload_in, r.mix, r.payload_out});
        enc.push_back(gf_gen_t{r.field, r.n_in, r.n_out, 0, (uint64_t)r.n_src, r.coef_in, r.mix, r.coef_out});
    }
    return gf_encode_plan_create(enc.data(), (int)enc.size(), GF_PATH_AUTO, plan);
}

extern "C" int gf_decode_plan_create(const gf_dec_t *gens, int n_gens, gf_plan_t **plan)
{
    if (!plan) return GF_EINVAL;
    *plan = nullptr;
    gf_plan *p = new gf_plan();
    p->kind = 1;
    int st = build_decode(gens, n_gens, p->dec);
    if (st != GF_OK) {
        delete p;
        return st;
    }
    const size_t x_total = align_up(p->dec.x_bytes, 256), r_total = align_up(p->dec.grow_bytes, 256);
    // descriptors do not depend on where X lands: size them with a
    // provisional placement, then allocate and place for real
    st = place_decode(p->dec, nullptr, nullptr);
    if (st != GF_OK) {
        delete p;
        return st;
    }
    const size_t stage = decode_stage_bytes(p->dec);
    if (decode_counters(p->dec) > kCounterBytes / sizeof(WorkCounter)) {
        delete p;
        return GF_EINVAL;
    }
    st = plan_alloc(p, kCounterBytes + x_total + r_total + stage);
    if (st != GF_OK) {
        delete p;
        return st;
    }
    char *dev_x = (char *)p->dev + kCounterBytes;
    st = place_decode(p->dec, dev_x, dev_x + x_total);
    if (st != GF_OK) {
        gf_plan_destroy(p);
        return st;
    }
    std::vector<char> host(stage + 16);
    const size_t end = stage_decode(p->dec, host.data(), (char *)p->dev + kCounterBytes + x_total + r_total, 0,
                                    reinterpret_cast<WorkCounter *>(p->dev));
    if (end && cudaMemcpy((char *)p->dev + kCounterBytes + x_total + r_total, host.data(), end,
                          cudaMemcpyHostToDevice) != cudaSuccess) {
        gf_plan_destroy(p);
        return GF_ECUDA;
    }
    *plan = p;
    return GF_OK;
}

extern "C" int gf_plan_launch(gf_plan_t *plan, gf_stream_t stream)
{
    if (!plan) return GF_EINVAL;
    if (plan->device != current_device()) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (plan->kind == 1) return launch_decode(plan->dec, s);
    for (const auto &b : plan->batches) {
        int st = launch_batch(b, s);
        if (st != GF_OK) return st;
    }
    return GF_OK;
}

extern "C" int gf_plan_kernel_count(const gf_plan_t *plan)
{
    if (!plan) return 0;
    int n = 0;
    const auto &bs = plan->kind == 1 ? plan->dec.batches : plan->batches;
    for (const auto &b : bs) n += b.total_tiles > 0 ? 1 : 0;
    if (plan->kind == 1 && !plan->dec.gens.empty()) n += 1;
    return n;
}

extern "C" int gf_plan_destroy(gf_plan_t *plan)
{
    if (!plan) return GF_OK;
    int st = GF_OK;
    if (plan->dev) {
        int prev = current_device();
        cudaSetDevice(plan->device);
        if (cudaDeviceSynchronize() != cudaSuccess) st = GF_ECUDA;
        cudaFree(plan->dev);
        cudaSetDevice(prev);
    }
    delete plan;
    return st;
}

// ---------------------------------------------------------------------------
// autotuner entry points
// ---------------------------------------------------------------------------
extern "C" int gf_autotune_encode(int field, int n_src, int n_coded, uint64_t len, int n_gens, gf_stream_t stream,
                                  int *out_path, int *out_variant)
{
    if (!field_ok(field) || n_src <= 0 || n_coded <= 0 || len == 0 || n_gens <= 0) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t src_b = (size_t)n_gens * n_src * len, coef_b = (size_t)n_gens * n_coded * n_src,
                 out_b = (size_t)n_gens * n_coded * len;
    uint8_t *buf = nullptr;
    if (cudaMalloc(&buf, src_b + coef_b + out_b) != cudaSuccess) {
        cudaGetLastError();
        return GF_ENOMEM;
    }
    fill_kernel<<<1024, 256, 0, s>>>(buf, src_b, 0x1234u, 0u);
    fill_kernel<<<1024, 256, 0, s>>>(buf + src_b, coef_b, 0x5678u, 1u << field);
    std::vector<gf_gen_t> gens(n_gens);
    for (int i = 0; i < n_gens; ++i) {
        gens[i] = gf_gen_t{field, n_src, n_coded, 0, len, buf + (size_t)i * n_src * len,
                           buf + src_b + (size_t)i * n_coded * n_src, buf + src_b + coef_b + (size_t)i * n_coded * len};
    }
    std::vector<TuneChoice> cands;
    if (bitsliced_available()) cands.push_back({GF_PATH_BITSLICED, 0});
    for (int v = 0; v < kNumTableVariants; ++v) cands.push_back({GF_PATH_TABLE, v});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TuneChoice pick{GF_PATH_TABLE, choose_table_variant(field, n_src, n_coded, len)};
    int st = GF_OK;
    t_last_tune.clear();
    for (const TuneChoice &c : cands) {
        t_force_variant = c.path == GF_PATH_TABLE ? c.variant : -1;
        float total = 0.f;
        int ok = GF_OK;
        for (int rep = 0; rep < 4 && ok == GF_OK; ++rep) {
            cudaEventRecord(e0, s);
            ok = gf_encode_batched_ex(gens.data(), n_gens, c.path, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) total += ms;  // first run is warm-up
        }
        t_force_variant = -1;
        if (ok != GF_OK) {
            if (ok == GF_ENOTSUP) continue;
            st = ok;
            break;
        }
        t_last_tune.emplace_back(c, total / 3.f);
        if (total < best) {
            best = total;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (st != GF_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[tune_key(field, n_src, n_coded, len)] = pick;
    }
    if (out_path) *out_path = pick.path;
    if (out_variant) *out_variant = pick.variant;
    return GF_OK;
}

extern "C" int gf_autotune_last(int cap, int *paths, int *variants, float *ms, int *n)
{
    if (cap < 0 || !n) return GF_EINVAL;
    *n = (int)t_last_tune.size();
    for (int i = 0; i < *n && i < cap; ++i) {
        if (paths) paths[i] = t_last_tune[i].first.path;
        if (variants) variants[i] = t_last_tune[i].first.variant;
        if (ms) ms[i] = t_last_tune[i].second;
    }
    return GF_OK;
}

extern "C" int gf_autotune_set(int field, int n_src, int n_coded, uint64_t len, int path, int variant)
{
    if (!field_ok(field) || (path != GF_PATH_TABLE && path != GF_PATH_BITSLICED)) return GF_EINVAL;
    if (variant < 0 || variant >= kNumTableVariants) return GF_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[tune_key(field, n_src, n_coded, len)] = TuneChoice{path, variant};
    return GF_OK;
}

extern "C" int gf_autotune_query(int field, int n_src, int n_coded, uint64_t len, int *path, int *variant)
{
    if (!field_ok(field)) return GF_EINVAL;
    const int p = choose_path(field, n_src, n_coded, len);
    if (path) *path = p;
    if (variant) *variant = p == GF_PATH_TABLE ? choose_table_variant(field, n_src, n_coded, len) : 0;
    return GF_OK;
}

extern "C" int gf_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    return GF_OK;
}

extern "C" int gf_autotune_save(const char *path)
{
    if (!path) return GF_EINVAL;
    FILE *f = fopen(path, "w");
    if (!f) return GF_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &kv : g_tune)
        fprintf(f, "%d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                std::get<3>(kv.first), kv.second.path, kv.second.variant);
    fclose(f);
    return GF_OK;
}

extern "C" int gf_autotune_load(const char *path)
{
    if (!path) return GF_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return GF_EINVAL;
    int a, b, c, d, pth, var;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    while (fscanf(f, "%d %d %d %d %d %d", &a, &b, &c, &d, &pth, &var) == 6) {
        if (!field_ok(a) || (pth != GF_PATH_TABLE && pth != GF_PATH_BITSLICED) || var < 0 ||
            var >= kNumTableVariants)
            continue;
        g_tune[TuneKey(a, b, c, d)] = TuneChoice{pth, var};
    }
    fclose(f);
    return GF_OK;
}
