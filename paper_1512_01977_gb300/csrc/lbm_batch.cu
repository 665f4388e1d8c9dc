// Batched stepping and the autotuners (include/lbm_axi_batch.h).
#include <string.h>

#include <new>
#include <vector>

#include "lbm_axi_batch.h"
#include "lbm_handle.h"
#include "lbm_launch.h"

using lbm::BatchSolve;
using lbm::Ops;

struct lbm_axi_batch {
    int n;
    int precision;
    bool mp, ax;
    int device;
    std::vector<lbm_axi*> solves;
    std::vector<int> cur0;  // each solve's current buffer when the batch was made
    void* d_solves;         // BatchSolve<R>[n]
    lbm::BatchTable<float>* h_table;  // FP32, n <= BatchTable::N: the descriptors as one kernel argument
    lbm::Tile* d_tiles;     // tile plan for (strip, grid)
    int* d_first;           // [ncta + 1]
    int ncta;
    int* d_err;             // [n]
    int* h_err;             // pinned [n]
    cudaStream_t stream;
    bool own_stream;
    long long steps;  // batch steps taken; parity = steps & 1
    int strip, grid;
    cudaGraphExec_t graph;  // two steps, parity 0 then 1
    int graph_strip, graph_grid;
    int pending;
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename R>
const Params<R>& params_of(const lbm_axi* h);
template <>
const Params<float>& params_of<float>(const lbm_axi* h) {
    return h->pf;
}
template <>
const Params<double>& params_of<double>(const lbm_axi* h) {
    return h->pdd;
}

template <typename R>
cudaError_t upload(lbm_axi_batch* b) {
    std::vector<BatchSolve<R>> hs(b->n);
    std::vector<int> nz(b->n), nr(b->n);
    for (int i = 0; i < b->n; i++) {
        lbm_axi* h = b->solves[i];
        hs[i].p = params_of<R>(h);
        hs[i].f_a = static_cast<const R*>(h->f[b->cur0[i]]);
        hs[i].f_b = static_cast<R*>(h->f[b->cur0[i] ^ 1]);
        nz[i] = h->nz;
        nr[i] = h->nr;
    }
    if constexpr (sizeof(R) == 4) {
        if (b->h_table)
            for (int i = 0; i < b->n; i++) b->h_table->s[i] = hs[i];
    }
    const int slots = b->grid > 0 ? b->grid : Ops<R>::batch_resident_ctas(b->strip);
    if (slots <= 0) return cudaErrorInvalidConfiguration;
    std::vector<lbm::Tile> tiles;
    std::vector<int> first;
    if (lbm::plan_tiles(nz.data(), nr.data(), b->n, b->strip, slots, tiles, first, nullptr) != LBM_OK)
        return cudaErrorMemoryAllocation;
    // the graph holds the old plan's pointers
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return e;
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_first) cudaFree(b->d_first);
    b->d_tiles = nullptr;
    b->d_first = nullptr;
    b->ncta = 0;
    e = cudaMalloc(&b->d_tiles, tiles.size() * sizeof(lbm::Tile));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_first, first.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_solves, hs.data(), sizeof(BatchSolve<R>) * b->n, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(lbm::Tile), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) b->ncta = (int)first.size() - 1;
    return e;
}

cudaError_t upload_tables(lbm_axi_batch* b) {
    return b->precision == 32 ? upload<float>(b) : upload<double>(b);
}

cudaError_t launch(lbm_axi_batch* b, int parity) {
    if (b->h_table)  // FP32, n <= BatchTable::N: parameters through the constant bank
        return Ops<float>::step_table(*b->h_table, b->d_tiles, b->d_first, b->ncta, b->mp, b->ax, parity, b->strip,
                                      b->d_err, b->stream);
    if (b->precision == 32)
        return Ops<float>::step_batch(static_cast<const BatchSolve<float>*>(b->d_solves), b->d_tiles, b->d_first,
                                      b->ncta, b->mp, b->ax, parity, b->strip, b->d_err, b->stream);
    return Ops<double>::step_batch(static_cast<const BatchSolve<double>*>(b->d_solves), b->d_tiles, b->d_first,
                                   b->ncta, b->mp, b->ax, parity, b->strip, b->d_err, b->stream);
}

int build_graph(lbm_axi_batch* b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    cudaError_t e = launch(b, 0);
    if (e == cudaSuccess) e = launch(b, 1);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        b->graph = nullptr;
        return LBM_ERR_CUDA;
    }
    b->graph_strip = b->strip;
    b->graph_grid = b->grid;
    return LBM_OK;
}

// Point every handle at the buffer holding its latest state.
void sync_handles(lbm_axi_batch* b) {
    for (int i = 0; i < b->n; i++) b->solves[i]->cur = b->cur0[i] ^ (int)(b->steps & 1);
}

void release(lbm_axi_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_solves) cudaFree(b->d_solves);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_first) cudaFree(b->d_first);
    if (b->d_err) cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b->h_table;
}

// Time `trials` launches of fn on stream s (ms per launch), non-destructively.
template <typename F>
float time_launches(cudaStream_t s, int trials, F&& fn) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    bool ok = fn() == cudaSuccess;  // warm-up launch
    ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
    for (int t = 0; t < trials && ok; t++) ok = fn() == cudaSuccess;
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = -1.f;
    if (ok) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms / trials : -1.f;
}

}  // namespace

extern "C" {

int lbm_axi_batch_create(lbm_axi* const* solves, int n, void* stream, lbm_axi_batch** out) {
    if (!out || !solves || n < 1) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    const lbm_axi* h0 = solves[0];
    if (!h0) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        const lbm_axi* h = solves[i];
        if (!h || !h->initialized || h->device != dev || h->precision != h0->precision ||
            h->nr < lbm::kStepMinRows || h->opts.multiphase != h0->opts.multiphase ||
            h->opts.axis_terms != h0->opts.axis_terms || unbatchable(h))
            return LBM_ERR_INVALID_ARG;
        for (int k = 0; k < i; k++)
            if (solves[k] == h) return LBM_ERR_INVALID_ARG;
    }
    lbm_axi_batch* b = new (std::nothrow) lbm_axi_batch;
    if (!b) return LBM_ERR_OOM;
    b->n = n;
    b->precision = h0->precision;
    b->mp = h0->opts.multiphase != 0;
    b->ax = h0->opts.axis_terms != 0;
    b->device = dev;
    b->d_solves = nullptr;
    b->h_table = nullptr;
    b->d_tiles = nullptr;
    b->d_first = nullptr;
    b->ncta = 0;
    b->d_err = nullptr;
    b->h_err = nullptr;
    b->stream = nullptr;
    b->own_stream = false;
    b->steps = 0;
    b->strip = lbm::kStripWide;
    b->grid = 0;
    b->graph = nullptr;
    b->graph_strip = b->graph_grid = -1;
    b->pending = LBM_OK;
    try {
        b->solves.assign(solves, solves + n);
        b->cur0.resize(n);
    } catch (...) {
        delete b;
        return LBM_ERR_OOM;
    }
    for (int i = 0; i < n; i++) {
        // finish whatever the solve's own stream was doing before the batch takes over
        if (cudaStreamSynchronize(solves[i]->stream) != cudaSuccess) {
            delete b;
            return LBM_ERR_CUDA;
        }
        b->cur0[i] = solves[i]->cur;
    }
    if (b->precision == 32 && n <= lbm::BatchTable<float>::N) {
        b->h_table = new (std::nothrow) lbm::BatchTable<float>();
        if (!b->h_table) {
            delete b;
            return LBM_ERR_OOM;
        }
    }
    const size_t ssz = b->precision == 32 ? sizeof(BatchSolve<float>) : sizeof(BatchSolve<double>);
    bool ok = cudaMalloc(&b->d_solves, ssz * n) == cudaSuccess &&
              cudaMalloc(&b->d_err, sizeof(int) * n) == cudaSuccess &&
              cudaMallocHost(&b->h_err, sizeof(int) * n) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(b);
        delete b;
        return LBM_ERR_OOM;
    }
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            release(b);
            delete b;
            return LBM_ERR_CUDA;
        }
        b->own_stream = true;
    }
    cudaError_t e = cudaMemsetAsync(b->d_err, 0, sizeof(int) * n, b->stream);
    if (e == cudaSuccess) e = upload_tables(b);
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

int lbm_axi_batch_step_async(lbm_axi_batch* b, long long nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
    DevGuard g(b->device);
    cudaError_t e = cudaSuccess;
    if (nsteps > 0 && (b->steps & 1)) {
        e = launch(b, 1);
        b->steps++;
        nsteps--;
    }
    if (e == cudaSuccess && nsteps >= 2) {
        if (!b->graph || b->graph_strip != b->strip || b->graph_grid != b->grid) {
            int rc = build_graph(b);
            if (rc != LBM_OK) return rc;
        }
        while (nsteps >= 2 && e == cudaSuccess) {
            e = cudaGraphLaunch(b->graph, b->stream);
            b->steps += 2;
            nsteps -= 2;
        }
    }
    if (e == cudaSuccess && nsteps == 1) {
        e = launch(b, 0);
        b->steps++;
    }
    sync_handles(b);
    if (e != cudaSuccess) {
        b->pending = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int lbm_axi_batch_status(lbm_axi_batch* b, int* status) {
    if (!b) return LBM_ERR_INVALID_ARG;
    DevGuard g(b->device);
    if (cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    int any = LBM_OK;
    for (int i = 0; i < b->n; i++) {
        const int s = b->h_err[i] ? LBM_ERR_UNPHYSICAL : LBM_OK;
        if (status) status[i] = s;
        if (s != LBM_OK) any = s;
    }
    return any;
}

int lbm_axi_batch_sync(lbm_axi_batch* b) {
    if (!b) return LBM_ERR_INVALID_ARG;
    int rc = lbm_axi_batch_status(b, nullptr);
    if (b->pending != LBM_OK) rc = b->pending;
    b->pending = LBM_OK;
    return rc;
}

int lbm_axi_batch_step(lbm_axi_batch* b, long long nsteps) {
    int rc = lbm_axi_batch_step_async(b, nsteps);
    if (rc != LBM_OK) {
        if (b && rc != LBM_ERR_INVALID_ARG) lbm_axi_batch_sync(b);
        return rc;
    }
    return lbm_axi_batch_sync(b);
}

int lbm_axi_batch_steps(const lbm_axi_batch* b, long long* steps) {
    if (!b || !steps) return LBM_ERR_INVALID_ARG;
    *steps = b->steps;
    return LBM_OK;
}

int lbm_axi_batch_get_tuning(const lbm_axi_batch* b, lbm_axi_batch_tuning* t) {
    if (!b || !t) return LBM_ERR_INVALID_ARG;
    t->strip = b->strip;
    t->grid = b->grid;
    return LBM_OK;
}

int lbm_axi_batch_set_tuning(lbm_axi_batch* b, const lbm_axi_batch_tuning* t) {
    if (!b || !t || (t->strip != lbm::kStripNarrow && t->strip != lbm::kStripWide) || t->grid < 0) return LBM_ERR_INVALID_ARG;
    DevGuard g(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (t->strip != b->strip || t->grid != b->grid || !b->d_tiles) {
        b->strip = t->strip;
        b->grid = t->grid;
        if (upload_tables(b) != cudaSuccess) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int lbm_axi_batch_autotune(lbm_axi_batch* b, int trials, lbm_axi_batch_tuning* chosen) {
    if (!b || trials < 1) return LBM_ERR_INVALID_ARG;
    DevGuard g(b->device);
    const int parity = (int)(b->steps & 1);
    float best = -1.f;
    lbm_axi_batch_tuning bt = {b->strip, b->grid};
    const int strips[2] = {lbm::kStripNarrow, lbm::kStripWide};
    // the solves' error words before the trials (trial results are discarded; a
    // solve that had already failed stays failed, and skipped, afterwards)
    if (cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    std::vector<int> err0;
    try {
        err0.assign(b->h_err, b->h_err + b->n);
    } catch (...) {
        return LBM_ERR_OOM;
    }
    for (int si = 0; si < 2; si++) {
        const int strip = strips[si];
        const int resident = b->precision == 32 ? Ops<float>::batch_resident_ctas(strip)
                                                : Ops<double>::batch_resident_ctas(strip);
        if (resident <= 0) continue;
        const int grids[2] = {0, 2 * resident};
        for (int gi = 0; gi < 2; gi++) {
            lbm_axi_batch_tuning t = {strip, grids[gi]};
            if (lbm_axi_batch_set_tuning(b, &t) != LBM_OK) return LBM_ERR_CUDA;
            const float ms = time_launches(b->stream, trials, [&] { return launch(b, parity); });
            if (ms > 0 && (best < 0 || ms < best)) {
                best = ms;
                bt.strip = strip;
                bt.grid = grids[gi];
            }
        }
    }
    if (best < 0) return LBM_ERR_CUDA;
    if (lbm_axi_batch_set_tuning(b, &bt) != LBM_OK) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(b->d_err, err0.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (chosen) *chosen = bt;
    return LBM_OK;
}

int lbm_axi_autotune(lbm_axi* h, int trials, lbm_axi_tuning* chosen) {
    if (!h || trials < 1) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DevGuard g(h->device);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    const int c = h->cur;
    float best = -1.f;
    lbm_axi_tuning bt = {h->path, h->rows_per_cta};
    auto fused = [&](int rows) {
        return h->precision == 32
                   ? Ops<float>::step(h->pf, (const float*)h->f[c], (float*)h->f[c ^ 1], rows, h->derr, h->stream)
                   : Ops<double>::step(h->pdd, (const double*)h->f[c], (double*)h->f[c ^ 1], rows, h->derr,
                                       h->stream);
    };
    auto split = [&]() {
        cudaError_t e;
        if (h->precision == 32) {
            const lbm::LinkPlanes<float> lk = link_planes<float>(h, c);
            e = Ops<float>::density(h->pf, (const float*)h->f[c], (float*)h->aux, h->derr, h->stream, lk);
            if (e == cudaSuccess)
                e = Ops<float>::update(h->pf, h->pdd, (const float*)h->f[c], (float*)h->f[c ^ 1],
                                       (const float*)h->aux, h->stream, lk, guo_of(h));
        } else {
            const lbm::LinkPlanes<double> lk = link_planes<double>(h, c);
            e = Ops<double>::density(h->pdd, (const double*)h->f[c], (double*)h->aux, h->derr, h->stream, lk);
            if (e == cudaSuccess)
                e = Ops<double>::update(h->pdd, h->pdd, (const double*)h->f[c], (double*)h->f[c ^ 1],
                                        (const double*)h->aux, h->stream, lk, guo_of(h));
        }
        return e;
    };
    if (fused_ok(h)) {
        // rows 0: the balanced wave over the tile plan (the form every collision variant has)
        const int rows_list[5] = {0, 32, 64, 144, 256};
        const int nrows = fv_of(h) ? 1 : 5;
        for (int q = 0; q < nrows; q++) {
            const float ms = time_launches(h->stream, trials, [&] {
                return rows_list[q] == 0 ? lbm_handle_step_tiles(h, c) : fused(rows_list[q]);
            });
            if (ms > 0 && (best < 0 || ms < best)) {
                best = ms;
                bt.path = LBM_PATH_FUSED;
                bt.rows_per_cta = rows_list[q];
            }
        }
    }
    const float ms = time_launches(h->stream, trials, split);
    if (ms > 0 && (best < 0 || ms < best)) {
        best = ms;
        bt.path = LBM_PATH_SPLIT;
        bt.rows_per_cta = h->rows_per_cta;
    }
    if (best < 0) return LBM_ERR_CUDA;
    if (cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int rc = lbm_axi_set_tuning(h, &bt);
    if (rc == LBM_OK && chosen) *chosen = bt;
    return rc;
}

void lbm_axi_batch_destroy(lbm_axi_batch* b) {
    if (!b) return;
    DevGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    sync_handles(b);
    release(b);
    delete b;
}

}  // extern "C"
