// Host runtime of the batched D1Q2 solver (lbrs_batch_* in include/lbrs.h).
//
// Many independent tubes share one workspace: two ping-pong copies of the
// concatenated distributions, tube tables (offset, length, 1/(2 lambda_b)) and
// a tile table.  A run advances tube b by steps[b]: tubes are ordered by
// decreasing steps so that the tubes still active after L*H steps form a
// prefix, their tiles are listed in that order, and launch L of the run
// covers the first active_tiles(L) tiles with up to H steps each
// (temporal blocking, lbrs_batch.cuh).  Tubes whose last launch left them in
// the other buffer are copied back by one final kernel.  The launch sequence
// of a run is captured once into a CUDA graph and replayed while the steps
// and the tuning stay the same.  An autotuner times one launch of each
// candidate (block size, cells per thread, H) on the current state and keeps
// the fastest per lattice update.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "lbrs.h"
#include "lbrs_batch.cuh"
#include "lbrs_launch.h"

using namespace lbrs;

namespace lbrs {
lbrs_status set_error(lbrs_status s, const char* msg);
}

namespace {

constexpr size_t kAlign = 256;
constexpr int kMinTile = 32;   // smallest tile any candidate uses; sizes the tile table

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BLayout {
    size_t f_bytes, f0, f1, tiles, copy_tiles, tube_off, tube_len, tube_steps, tube_c, tube_lam, total;
    int64_t max_tiles;
};

int64_t total_cells(const lbrs_batch_config* c)
{
    int64_t n = 0;
    for (int64_t b = 0; b < c->batch; ++b) n += c->lengths[b];
    return n;
}

BLayout layout_of(const lbrs_batch_config* c)
{
    BLayout L;
    const size_t elem = c->precision == LBRS_F64 ? 8 : 4;
    const int64_t N = total_cells(c);
    L.max_tiles = N / kMinTile + c->batch + 1;
    L.f_bytes = (size_t)N * 3 * (c->lattice == LBRS_D1Q3 ? 3 : 2) * elem;
    size_t off = 0;
    L.f0 = off;
    off += align_up(L.f_bytes);
    L.f1 = off;
    off += align_up(L.f_bytes);
    L.tiles = off;
    off += align_up((size_t)L.max_tiles * sizeof(BatchTile));
    L.copy_tiles = off;
    off += align_up((size_t)L.max_tiles * sizeof(BatchTile));
    L.tube_off = off;
    off += align_up((size_t)c->batch * sizeof(int64_t));
    L.tube_len = off;
    off += align_up((size_t)c->batch * sizeof(int));
    L.tube_steps = off;
    off += align_up((size_t)c->batch * sizeof(int));
    L.tube_c = off;
    off += align_up((size_t)c->batch * elem);
    L.tube_lam = off;
    off += align_up((size_t)c->batch * sizeof(double));
    L.total = off;
    return L;
}

}  // namespace

struct lbrs_batch {
    lbrs_batch_config cfg;
    std::vector<int64_t> lengths;
    std::vector<double> lambda;
    BLayout L;
    int64_t N;
    int f64;
    int q;                   // populations per field: 2 (D1Q2) or 3 (D1Q3)
    char* ws;
    char* f[2];
    int cur;
    bool has_state;
    cudaStream_t stream;
    lbrs_batch_tuning tuning;
    int64_t launches;
    // cached plan and graph of the last run
    std::vector<int64_t> plan_steps;
    lbrs_batch_tuning plan_tuning;
    int plan_cur;
    int plan_nlaunch;
    cudaGraphExec_t graph;
    cudaStream_t cap_stream;
    char err[512];
};

namespace {

lbrs_status bfail(lbrs_batch* B, lbrs_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (B) snprintf(B->err, sizeof B->err, "%s", buf);
    return set_error(s, buf);
}

#define BCUDA(B, call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return bfail((B), LBRS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

lbrs_status validate(const lbrs_batch_config* c)
{
    if (!c) return bfail(nullptr, LBRS_EINVAL, "config is NULL");
    if (c->struct_size != sizeof(lbrs_batch_config))
        return bfail(nullptr, LBRS_EINVAL, "config.struct_size %u != sizeof(lbrs_batch_config) %zu", c->struct_size,
                     sizeof(lbrs_batch_config));
    if (c->precision != LBRS_F64 && c->precision != LBRS_F32) return bfail(nullptr, LBRS_EINVAL, "unknown precision");
    if (c->lattice != LBRS_D1Q2 && c->lattice != LBRS_D1Q3)
        return bfail(nullptr, LBRS_EINVAL, "batched tubes are D1Q2 or D1Q3");
    if (c->boundary != LBRS_BC_TRANSMISSIVE && c->boundary != LBRS_BC_PERIODIC)
        return bfail(nullptr, LBRS_EINVAL, "batched tubes support transmissive or periodic ends");
    if (c->batch < 1 || c->batch > (1 << 30)) return bfail(nullptr, LBRS_EINVAL, "batch must be in [1, 2^30]");
    if (!c->lengths || !c->lambda) return bfail(nullptr, LBRS_EINVAL, "lengths and lambda are required");
    int64_t n = 0;
    for (int64_t b = 0; b < c->batch; ++b) {
        if (c->lengths[b] < 1 || c->lengths[b] > (1 << 30)) return bfail(nullptr, LBRS_EINVAL, "tube %lld: bad length", (long long)b);
        if (!(c->lambda[b] > 0.0) || !isfinite(c->lambda[b])) return bfail(nullptr, LBRS_EINVAL, "tube %lld: lambda must be positive", (long long)b);
        n += c->lengths[b];
    }
    if (n > (1LL << 40)) return bfail(nullptr, LBRS_EINVAL, "too many cells");
    if (!(c->gamma > 1.0) || !isfinite(c->gamma)) return bfail(nullptr, LBRS_EINVAL, "gamma must be > 1");
    if (!(c->omega > 0.0 && c->omega < 2.0)) return bfail(nullptr, LBRS_EINVAL, "omega must lie in (0, 2)");
    return LBRS_OK;
}

bool tuning_ok(const lbrs_batch_tuning& t)
{
    if (t.block != 128 && t.block != 256 && t.block != 512) return false;
    if (t.cells_per_thread < 1 || t.cells_per_thread > 8) return false;
    if (t.halo < 1 || t.halo > 256) return false;
    const int tile = t.block * t.cells_per_thread - 2 * t.halo;
    return tile >= kMinTile;
}

int tile_of(const lbrs_batch_tuning& t) { return t.block * t.cells_per_thread - 2 * t.halo; }

constexpr size_t kMaxSmem = 227 * 1024;

size_t smem_of(const lbrs_batch* B, const lbrs_batch_tuning& t)
{
    return 2 * 3 * (size_t)B->q * (size_t)(tile_of(t) + 2 * t.halo) * (B->f64 ? 8 : 4);
}

cudaError_t prepare(const lbrs_batch* B, const lbrs_batch_tuning& t)
{
    return B->f64 ? prepare_batch_f64(t.block, smem_of(B, t), B->q) : prepare_batch_f32(t.block, smem_of(B, t), B->q);
}

// Tubes ordered by decreasing steps (stable) and their tiles in that order.
// active[L] = tiles of tubes with steps > L*H.
void plan(const lbrs_batch* B, const int64_t* steps, const lbrs_batch_tuning& t, std::vector<BatchTile>& tiles,
          std::vector<int>& active, int& nlaunch)
{
    const int64_t nb = B->cfg.batch;
    const int tile = tile_of(t), H = t.halo;
    std::vector<int64_t> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return steps[a] > steps[b]; });
    tiles.clear();
    std::vector<int64_t> tube_end_tile(nb);
    for (int64_t r = 0; r < nb; ++r) {
        const int64_t b = order[r];
        if (steps[b] > 0)
            for (int64_t x = 0; x < B->lengths[b]; x += tile)
                tiles.push_back(BatchTile{(int)b, (int)x, (int)std::min<int64_t>(tile, B->lengths[b] - x), 0});
        tube_end_tile[r] = (int64_t)tiles.size();
    }
    const int64_t max_steps = steps[order[0]];
    nlaunch = (int)((max_steps + H - 1) / H);
    active.assign(nlaunch, 0);
    // the tubes with steps > L*H are a prefix of the order, longer as L falls
    int64_t cnt = 0;
    for (int L = nlaunch - 1; L >= 0; --L) {
        while (cnt < nb && steps[order[cnt]] > (int64_t)L * H) ++cnt;
        active[L] = cnt ? (int)tube_end_tile[cnt - 1] : 0;
    }
}

template <typename T>
BatchArgs<T> batch_args(const lbrs_batch* B, int from, const lbrs_batch_tuning& t, int launch)
{
    BatchArgs<T> a{};
    a.src = (const T*)B->f[from];
    a.dst = (T*)B->f[from ^ 1];
    a.N = B->N;
    a.tiles = (const BatchTile*)(B->ws + B->L.tiles);
    a.tube_off = (const int64_t*)(B->ws + B->L.tube_off);
    a.tube_len = (const int*)(B->ws + B->L.tube_len);
    a.tube_steps = (const int*)(B->ws + B->L.tube_steps);
    a.tube_c = (const T*)(B->ws + B->L.tube_c);
    a.tile_cells = tile_of(t);
    a.halo = t.halo;
    a.periodic = B->cfg.boundary == LBRS_BC_PERIODIC;
    a.launch = launch;
    a.q = B->q;
    a.om = (T)B->cfg.omega;
    a.om1 = (T)(1.0 - B->cfg.omega);
    a.gm1 = (T)(B->cfg.gamma - 1.0);
    return a;
}

cudaError_t launch_one(lbrs_batch* B, int from, const lbrs_batch_tuning& t, int launch, int ntiles, cudaStream_t s)
{
    if (B->f64) return launch_batch_f64(batch_args<double>(B, from, t, launch), ntiles, t.block, s);
    return launch_batch_f32(batch_args<float>(B, from, t, launch), ntiles, t.block, s);
}

// Upload the tube steps and the tile tables of a run; returns the launch plan.
lbrs_status upload_plan(lbrs_batch* B, const int64_t* steps, const lbrs_batch_tuning& t, std::vector<int>& active,
                        int& nlaunch, int& ncopy, int& final_parity)
{
    std::vector<BatchTile> tiles;
    plan(B, steps, t, tiles, active, nlaunch);
    if ((int64_t)tiles.size() > B->L.max_tiles) return bfail(B, LBRS_EINVAL, "tile table overflow");
    std::vector<int> st(B->cfg.batch);
    for (int64_t b = 0; b < B->cfg.batch; ++b) st[b] = (int)steps[b];
    final_parity = (B->cur + nlaunch) & 1;
    // tubes whose last launch left them in the other buffer
    std::vector<BatchTile> copies;
    for (int64_t b = 0; b < B->cfg.batch; ++b) {
        const int64_t nl = (steps[b] + t.halo - 1) / t.halo;
        if (((B->cur + nl) & 1) != final_parity)
            for (int64_t x = 0; x < B->lengths[b]; x += 4096)
                copies.push_back(BatchTile{(int)b, (int)x, (int)std::min<int64_t>(4096, B->lengths[b] - x), 0});
    }
    if ((int64_t)copies.size() > B->L.max_tiles) return bfail(B, LBRS_EINVAL, "copy table overflow");
    ncopy = (int)copies.size();
    BCUDA(B, cudaMemcpyAsync(B->ws + B->L.tube_steps, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice,
                             B->stream));
    if (!tiles.empty())
        BCUDA(B, cudaMemcpyAsync(B->ws + B->L.tiles, tiles.data(), tiles.size() * sizeof(BatchTile),
                                 cudaMemcpyHostToDevice, B->stream));
    if (!copies.empty())
        BCUDA(B, cudaMemcpyAsync(B->ws + B->L.copy_tiles, copies.data(), copies.size() * sizeof(BatchTile),
                                 cudaMemcpyHostToDevice, B->stream));
    BCUDA(B, cudaStreamSynchronize(B->stream));   // host vectors die on return
    return LBRS_OK;
}

cudaError_t enqueue_run(lbrs_batch* B, const lbrs_batch_tuning& t, const std::vector<int>& active, int nlaunch,
                        int ncopy, int final_parity, cudaStream_t s)
{
    int from = B->cur;
    for (int L = 0; L < nlaunch; ++L) {
        cudaError_t e = launch_one(B, from, t, L, active[L], s);
        if (e != cudaSuccess) return e;
        from ^= 1;
    }
    if (ncopy > 0) {
        const void* src = B->f[final_parity ^ 1];
        void* dst = B->f[final_parity];
        const BatchTile* ct = (const BatchTile*)(B->ws + B->L.copy_tiles);
        const int64_t* off = (const int64_t*)(B->ws + B->L.tube_off);
        return B->f64 ? launch_batch_copy_f64((const double*)src, (double*)dst, B->N, ct, ncopy, off, 3 * B->q, s)
                      : launch_batch_copy_f32((const float*)src, (float*)dst, B->N, ct, ncopy, off, 3 * B->q, s);
    }
    return cudaSuccess;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

lbrs_status lbrs_batch_workspace_size(const lbrs_batch_config* cfg, size_t* bytes)
{
    if (!bytes) return bfail(nullptr, LBRS_EINVAL, "bytes is NULL");
    lbrs_status st = validate(cfg);
    if (st != LBRS_OK) return st;
    *bytes = layout_of(cfg).total;
    return LBRS_OK;
}

lbrs_status lbrs_batch_create(const lbrs_batch_config* cfg, void* d_workspace, size_t bytes, lbrs_batch** out)
{
    if (!out) return bfail(nullptr, LBRS_EINVAL, "out is NULL");
    *out = nullptr;
    lbrs_status st = validate(cfg);
    if (st != LBRS_OK) return st;
    const BLayout L = layout_of(cfg);
    if (!d_workspace || (uintptr_t)d_workspace % kAlign)
        return bfail(nullptr, LBRS_EINVAL, "workspace NULL or not 256-byte aligned");
    if (bytes < L.total) return bfail(nullptr, LBRS_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, L.total);
    lbrs_batch* B = new (std::nothrow) lbrs_batch();
    if (!B) return bfail(nullptr, LBRS_ENOMEM, "host allocation failed");
    B->cfg = *cfg;
    B->lengths.assign(cfg->lengths, cfg->lengths + cfg->batch);
    B->lambda.assign(cfg->lambda, cfg->lambda + cfg->batch);
    B->cfg.lengths = B->lengths.data();
    B->cfg.lambda = B->lambda.data();
    B->L = L;
    B->N = total_cells(cfg);
    B->f64 = cfg->precision == LBRS_F64;
    B->q = cfg->lattice == LBRS_D1Q3 ? 3 : 2;
    B->ws = (char*)d_workspace;
    B->f[0] = B->ws + L.f0;
    B->f[1] = B->ws + L.f1;
    B->stream = (cudaStream_t)cfg->cuda_stream;
    B->tuning = lbrs_batch_tuning{256, 2, 16, 0};
    // tube tables
    std::vector<int64_t> off(cfg->batch);
    std::vector<int> len(cfg->batch);
    int64_t o = 0;
    for (int64_t b = 0; b < cfg->batch; ++b) {
        off[b] = o;
        len[b] = (int)cfg->lengths[b];
        o += cfg->lengths[b];
    }
    cudaError_t e = cudaMemcpyAsync(B->ws + L.tube_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->ws + L.tube_len, len.data(), len.size() * 4, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->ws + L.tube_lam, B->lambda.data(), B->lambda.size() * 8, cudaMemcpyHostToDevice,
                            B->stream);
    if (e == cudaSuccess) {
        if (B->f64) {
            std::vector<double> c(cfg->batch);
            for (int64_t b = 0; b < cfg->batch; ++b) c[b] = 1.0 / (2.0 * cfg->lambda[b]);
            e = cudaMemcpyAsync(B->ws + L.tube_c, c.data(), c.size() * 8, cudaMemcpyHostToDevice, B->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        } else {
            std::vector<float> c(cfg->batch);
            for (int64_t b = 0; b < cfg->batch; ++b) c[b] = (float)(1.0 / (2.0 * cfg->lambda[b]));
            e = cudaMemcpyAsync(B->ws + L.tube_c, c.data(), c.size() * 4, cudaMemcpyHostToDevice, B->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        }
    }
    if (e != cudaSuccess) {
        lbrs_status s = bfail(nullptr, LBRS_ECUDA, "uploading tube tables: %s", cudaGetErrorString(e));
        delete B;
        return s;
    }
    *out = B;
    return LBRS_OK;
}

void lbrs_batch_destroy(lbrs_batch* B)
{
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    delete B;
}

lbrs_status lbrs_batch_set_state(lbrs_batch* B, const void* W, int on_device, int dtype, int kind)
{
    if (!B) return bfail(nullptr, LBRS_EINVAL, "batch is NULL");
    if (!W) return bfail(B, LBRS_EINVAL, "W is NULL");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return bfail(B, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    if (kind != LBRS_CONSERVED && kind != LBRS_PRIMITIVE) return bfail(B, LBRS_EINVAL, "unknown state kind");
    // f = f^eq(U(W)) with each cell's own tube lambda (the kernel finds the tube
    // of a cell by bisection in the offset table)
    const void* src = W;
    const size_t wbytes = (size_t)3 * B->N * (dtype == LBRS_F64 ? 8 : 4);
    if (!on_device) {
        char* stage = B->f[B->cur ^ 1];
        BCUDA(B, cudaMemcpyAsync(stage, W, wbytes, cudaMemcpyHostToDevice, B->stream));
        src = stage;
    }
    BCUDA(B, launch_batch_set_state(B->f64, src, dtype == LBRS_F32, kind, B->f[B->cur], B->N,
                                    (const int64_t*)(B->ws + B->L.tube_off), B->cfg.batch,
                                    (const double*)(B->ws + B->L.tube_lam), B->cfg.gamma, B->q, B->stream));
    B->launches += 1;
    if (!on_device) BCUDA(B, cudaStreamSynchronize(B->stream));
    B->has_state = true;
    return LBRS_OK;
}

lbrs_status lbrs_batch_get_tuning(const lbrs_batch* B, lbrs_batch_tuning* t)
{
    if (!B || !t) return bfail(nullptr, LBRS_EINVAL, "NULL argument");
    *t = B->tuning;
    return LBRS_OK;
}

lbrs_status lbrs_batch_set_tuning(lbrs_batch* B, const lbrs_batch_tuning* t)
{
    if (!B || !t) return bfail(nullptr, LBRS_EINVAL, "NULL argument");
    if (!tuning_ok(*t) || smem_of(B, *t) > kMaxSmem)
        return bfail(B, LBRS_EINVAL, "invalid tuning (block %d, cells/thread %d, halo %d)", t->block,
                     t->cells_per_thread, t->halo);
    B->tuning = *t;
    return LBRS_OK;
}

lbrs_status lbrs_batch_run(lbrs_batch* B, const int64_t* steps)
{
    NvtxRange range("lbrs_batch_run");
    if (!B) return bfail(nullptr, LBRS_EINVAL, "batch is NULL");
    if (!steps) return bfail(B, LBRS_EINVAL, "steps is NULL");
    if (!B->has_state) return bfail(B, LBRS_ESTATE, "no state set");
    int64_t max_steps = 0;
    for (int64_t b = 0; b < B->cfg.batch; ++b) {
        if (steps[b] < 0 || steps[b] > (1 << 30)) return bfail(B, LBRS_EINVAL, "tube %lld: bad step count", (long long)b);
        max_steps = std::max(max_steps, steps[b]);
    }
    if (max_steps == 0) return LBRS_OK;
    const lbrs_batch_tuning t = B->tuning;
    const bool same = B->graph && B->plan_cur == B->cur && !memcmp(&B->plan_tuning, &t, sizeof t) &&
                      B->plan_steps.size() == (size_t)B->cfg.batch &&
                      std::equal(B->plan_steps.begin(), B->plan_steps.end(), steps);
    int final_parity;
    if (same) {
        BCUDA(B, cudaGraphLaunch(B->graph, B->stream));
        final_parity = (B->cur + B->plan_nlaunch) & 1;
        B->launches += B->plan_nlaunch + 1;
    } else {
        std::vector<int> active;
        int nlaunch, ncopy;
        lbrs_status st = upload_plan(B, steps, t, active, nlaunch, ncopy, final_parity);
        if (st != LBRS_OK) return st;
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        if (!B->cap_stream) BCUDA(B, cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
        BCUDA(B, prepare(B, t));
        BCUDA(B, cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = enqueue_run(B, t, active, nlaunch, ncopy, final_parity, B->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(B->cap_stream, &g);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(B, LBRS_ECUDA, "capturing the run: %s",
                         cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        cudaError_t ie = cudaGraphInstantiate(&B->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            B->graph = nullptr;
            return bfail(B, LBRS_ECUDA, "instantiating the run graph: %s", cudaGetErrorString(ie));
        }
        B->plan_steps.assign(steps, steps + B->cfg.batch);
        B->plan_tuning = t;
        B->plan_cur = B->cur;
        B->plan_nlaunch = nlaunch;
        BCUDA(B, cudaGraphLaunch(B->graph, B->stream));
        B->launches += nlaunch + (ncopy > 0);
    }
    B->cur = final_parity;
    return LBRS_OK;
}

lbrs_status lbrs_batch_autotune(lbrs_batch* B, const int64_t* steps, lbrs_batch_tuning* chosen, double* ns_per_update)
{
    if (!B) return bfail(nullptr, LBRS_EINVAL, "batch is NULL");
    if (!steps) return bfail(B, LBRS_EINVAL, "steps is NULL");
    if (!B->has_state) return bfail(B, LBRS_ESTATE, "no state set");
    static const int blocks[] = {128, 256, 512};
    static const int cpts[] = {1, 2, 4, 8};
    static const int halos[] = {8, 16, 32, 64};
    cudaEvent_t e0, e1;
    BCUDA(B, cudaEventCreate(&e0));
    BCUDA(B, cudaEventCreate(&e1));
    double best = 1e300;
    lbrs_batch_tuning best_t = B->tuning;
    lbrs_status result = LBRS_OK;
    for (int bi : blocks)
        for (int ci : cpts)
            for (int hi : halos) {
                lbrs_batch_tuning t{bi, ci, hi, 0};
                if (!tuning_ok(t) || smem_of(B, t) > kMaxSmem) continue;
                if (prepare(B, t) != cudaSuccess) continue;
                std::vector<int> active;
                int nlaunch, ncopy, fp;
                lbrs_status st = upload_plan(B, steps, t, active, nlaunch, ncopy, fp);
                if (st != LBRS_OK) {
                    result = st;
                    break;
                }
                // lattice updates of launch 0: every tile of a tube with steps > 0, min(H, steps) steps
                double lups = 0.0;
                for (int64_t b = 0; b < B->cfg.batch; ++b)
                    lups += (double)B->lengths[b] * (double)std::min<int64_t>(t.halo, steps[b]);
                cudaError_t e = launch_one(B, B->cur, t, 0, active.empty() ? 0 : active[0], B->stream);   // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, B->stream);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_one(B, B->cur, t, 0, active[0], B->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    result = bfail(B, LBRS_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
                    break;
                }
                const double per = ms * 1e6 / 3.0 / lups;
                if (per < best) {
                    best = per;
                    best_t = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != LBRS_OK) return result;
    if (B->graph) {               // the tile table now holds the last candidate's plan
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    B->tuning = best_t;
    if (chosen) *chosen = best_t;
    if (ns_per_update) *ns_per_update = best;
    return LBRS_OK;
}

lbrs_status lbrs_batch_moments(lbrs_batch* B, void* U_out, int on_device, int dtype)
{
    if (!B) return bfail(nullptr, LBRS_EINVAL, "batch is NULL");
    if (!U_out) return bfail(B, LBRS_EINVAL, "U_out is NULL");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return bfail(B, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    if (!B->has_state) return bfail(B, LBRS_ESTATE, "no state set");
    void* dst = on_device ? U_out : (void*)B->f[B->cur ^ 1];
    BCUDA(B, launch_moments(B->q == 3 ? LAT_D1Q3 : LAT_D1Q2, B->f64, B->f[B->cur], dst, dtype == LBRS_F32, B->N,
                            B->N, B->stream));
    B->launches += 1;
    if (!on_device) {
        BCUDA(B, cudaMemcpyAsync(U_out, dst, (size_t)3 * B->N * (dtype == LBRS_F64 ? 8 : 4), cudaMemcpyDeviceToHost,
                                 B->stream));
        BCUDA(B, cudaStreamSynchronize(B->stream));
    }
    return LBRS_OK;
}

lbrs_status lbrs_batch_get_distributions(lbrs_batch* B, void* dst, int on_device)
{
    if (!B || !dst) return bfail(B, LBRS_EINVAL, "NULL argument");
    if (!B->has_state) return bfail(B, LBRS_ESTATE, "no state set");
    BCUDA(B, cudaMemcpyAsync(dst, B->f[B->cur], B->L.f_bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, B->stream));
    if (!on_device) BCUDA(B, cudaStreamSynchronize(B->stream));
    return LBRS_OK;
}

lbrs_status lbrs_batch_launch_count(const lbrs_batch* B, int64_t* launches)
{
    if (!B || !launches) return bfail(nullptr, LBRS_EINVAL, "NULL argument");
    *launches = B->launches;
    return LBRS_OK;
}

const char* lbrs_batch_last_error(const lbrs_batch* B) { return B ? B->err : ""; }

}  // extern "C"
