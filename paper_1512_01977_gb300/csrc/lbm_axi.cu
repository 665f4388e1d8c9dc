// C ABI of the engine (include/lbm_axi.h): handle lifetime, device memory,
// the step loop (replayed as CUDA-graph chunks), moments and FP64 reductions.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbm_axi.h"
#include "lbm_eos_host.h"
#include "lbm_launch.h"

using lbm::Ops;
using lbm::Params;

namespace {

void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_release)(void*, void*) = nullptr;
void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
    void* p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void dev_free(void* p, bool via_hook, void* ctx, void (*release)(void*, void*)) {
    if (!p) return;
    if (via_hook) release(p, ctx);
    else cudaFree(p);
}

int pitch_of(int nz) { return (nz + 31) / 32 * 32; }

}  // namespace

#include "lbm_handle.h"

// The balanced one-wave grid: the fused kernel over this solve's tile plan, its
// descriptor passed by value; the same arithmetic as inside any batch.
cudaError_t lbm_handle_step_tiles(lbm_axi* h, int c) {
    const bool mp = h->opts.multiphase != 0, ax = h->opts.axis_terms != 0;
    if (h->precision == 32) {
        const lbm::BatchSolve<float> d{h->pf, (const float*)h->f[0], (float*)h->f[1], (const float*)h->hb[0],
                                       (float*)h->hb[1]};
        return Ops<float>::step_single(d, h->d_tiles, h->d_first, h->ncta, mp, ax, c, h->derr, h->stream, fv_of(h));
    }
    const lbm::BatchSolve<double> d{h->pdd, (const double*)h->f[0], (double*)h->f[1], (const double*)h->hb[0],
                                    (double*)h->hb[1]};
    return Ops<double>::step_single(d, h->d_tiles, h->d_first, h->ncta, mp, ax, c, h->derr, h->stream, fv_of(h));
}

namespace {

template <typename R>
Params<R> make_params(const lbm_axi* h) {
    Params<R> p;
    p.nz = h->nz;
    p.nr = h->nr;
    p.pitch = h->pitch;
    p.axis_a = (R)(h->opts.axis_a_term == LBM_AXIS_A_EXPANSION ? 2.0 : 6.0);
    p.plane = h->plane;
    p.tau_inv = (R)(1.0 / h->tau);
    p.nu = (R)((h->tau - 0.5) / 3.0);
    p.A = (R)h->A;
    p.rho_ref = (R)h->opts.rho_ref;
    p.gz = (R)h->opts.g_z;
    p.eos = h->eos.kind;
    p.T = (R)h->T;
    p.a = (R)h->eos.a;
    p.b = (R)h->eos.b;
    p.Rg = (R)h->eos.R;
    p.lambda = (R)h->eos.lambda;
    p.top = h->opts.top_bc;
    p.axis = h->opts.axis_terms;
    p.multiphase = h->opts.multiphase;
    p.kappa = h->opts.kappa_mode;
    p.hr_sign = h->opts.hr_sign;
    return p;
}

// The FP64 copy used for outputs (moments' P_k, pressure jump) carries the
// reference density as stored in the arithmetic type of the populations.
Params<double> make_params_out(const lbm_axi* h) {
    Params<double> pd = make_params<double>(h);
    if (h->precision == 32) pd.rho_ref = (double)(float)h->opts.rho_ref;
    return pd;
}

double stored_rho_ref(const lbm_axi* h) {
    return h->precision == 32 ? (double)(float)h->opts.rho_ref : h->opts.rho_ref;
}

// One step.  Fused path: kernel (b') reads f[cur] and writes f[cur^1].  Split
// path: kernel (a) on the current populations, kernel (b) into the other buffer.
cudaError_t enqueue_step(lbm_axi* h) {
    const int c = h->cur;
    cudaError_t e;
    if (h->path == LBM_PATH_FUSED && h->rows_per_cta == 0) {
        e = lbm_handle_step_tiles(h, c);
        h->cur = c ^ 1;
        return e;
    }
    if (h->path == LBM_PATH_FUSED) {
        if (h->precision == 32)
            e = Ops<float>::step(h->pf, (const float*)h->f[c], (float*)h->f[c ^ 1], h->rows_per_cta, h->derr,
                                 h->stream);
        else
            e = Ops<double>::step(h->pdd, (const double*)h->f[c], (double*)h->f[c ^ 1], h->rows_per_cta, h->derr,
                                  h->stream);
        h->cur = c ^ 1;
        return e;
    }
    if (h->precision == 32) {
        const lbm::LinkPlanes<float> lk = link_planes<float>(h, c);
        e = Ops<float>::density(h->pf, (const float*)h->f[c], (float*)h->aux, h->derr, h->stream, lk);
        if (e == cudaSuccess)
            e = Ops<float>::update(h->pf, h->pdd, (const float*)h->f[c], (float*)h->f[c ^ 1], (const float*)h->aux,
                                   h->stream, lk, guo_of(h));
    } else {
        const lbm::LinkPlanes<double> lk = link_planes<double>(h, c);
        e = Ops<double>::density(h->pdd, (const double*)h->f[c], (double*)h->aux, h->derr, h->stream, lk);
        if (e == cudaSuccess)
            e = Ops<double>::update(h->pdd, h->pdd, (const double*)h->f[c], (double*)h->f[c ^ 1],
                                    (const double*)h->aux, h->stream, lk, guo_of(h));
    }
    h->cur = c ^ 1;
    return e;
}

cudaError_t enqueue_density(lbm_axi* h) {
    if (h->precision == 32)
        return Ops<float>::density(h->pf, (const float*)h->f[h->cur], (float*)h->aux, h->derr, h->stream,
                                   link_planes<float>(h, h->cur));
    return Ops<double>::density(h->pdd, (const double*)h->f[h->cur], (double*)h->aux, h->derr, h->stream,
                                link_planes<double>(h, h->cur));
}

// Graph of an even number of steps starting and ending in buffer 0.
int build_graph(lbm_axi* h, int steps) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    const int saved = h->cur;
    h->cur = 0;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < steps && e == cudaSuccess; s++) e = enqueue_step(h);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    h->cur = saved;
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        h->graph = nullptr;
        return LBM_ERR_CUDA;
    }
    h->graph_steps = steps;
    return LBM_OK;
}

// Steps per graph replay: enough work per launch for tiny grids, at least 2.
int chunk_steps(const lbm_axi* h) {
    const long long cells = (long long)h->nz * h->nr;
    long long c = (4LL << 20) / (cells > 0 ? cells : 1);
    if (c < 2) c = 2;
    if (c > 256) c = 256;
    return (int)(c & ~1LL);
}

int read_error(lbm_axi* h) {
    if (cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    return *h->herr ? LBM_ERR_UNPHYSICAL : LBM_OK;
}

// Bare velocity of a state whose physical velocity is to be u:
// the solve holds f^eq(rho, u) and (pz, pr) its physical velocity
// u + F/(2 rho), so u0 = u - F/(2 rho) = 2 u - (pz, pr), written over (pz, pr).
__global__ void __launch_bounds__(256) k_bare_from_physical(long long n, const double* __restrict__ uz,
                                                           const double* __restrict__ ur, double* __restrict__ pz,
                                                           double* __restrict__ pr) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double vz = uz ? uz[c] : 0.0, vr = ur ? ur[c] : 0.0;
    pz[c] = vz - (pz[c] - vz);
    pr[c] = vr - (pr[c] - vr);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void release_all(lbm_axi* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    dev_free(h->f[0], h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->f[1], h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->aux, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->mout, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->partial, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->dred, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->derr, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->d_tiles, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->d_first, h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->hb[0], h->via_hook, h->hook_ctx, h->hook_release);
    dev_free(h->hb[1], h->via_hook, h->hook_ctx, h->hook_release);
    if (h->herr) cudaFreeHost(h->herr);
    if (h->hred) cudaFreeHost(h->hred);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

extern "C" {

void lbm_axi_default_opts(lbm_axi_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = 64;
    o->top_bc = LBM_TOP_FREESLIP;
    o->axis_terms = 1;
    o->multiphase = 1;
    o->kappa_mode = LBM_KAPPA_THERMO;
    o->hr_sign = -1;
    o->rho_ref = 0.0;
    o->g_z = 0.0;
    o->stream = nullptr;
    o->h_eval = LBM_H_LOCAL;
    o->forcing = LBM_FORCING_EDM;
    o->axis_a_term = LBM_AXIS_A_PRINTED;
}

size_t lbm_axi_footprint(int nz, int nr, int precision) {
    if (nz < 1 || nr < 1) return 0;
    const size_t s = precision == 32 ? 4 : 8;
    const size_t plane = (size_t)pitch_of(nz) * nr;
    return 2 * 9 * plane * s + 4 * plane * s + 4 * (size_t)nz * nr * 8 + 4 * lbm::kReduceBlocks * 8 + 64;
}

int lbm_axi_create(int nz, int nr, double tau, const lbm_eos* eos, double A, const lbm_axi_opts* opts,
                   lbm_axi** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    lbm_axi_opts o;
    if (opts) o = *opts;
    else lbm_axi_default_opts(&o);
    if (nz < 1 || nr < 1 || (long long)nz * nr > (1LL << 31) / 16) return LBM_ERR_INVALID_ARG;
    // the step kernels index a population buffer (9 planes of pitch x nr) with 32-bit offsets
    if (9LL * pitch_of(nz) * nr >= (1LL << 31)) return LBM_ERR_INVALID_ARG;
    if (!(tau > 0.5) || !(tau < 1e6)) return LBM_ERR_INVALID_ARG;
    if (o.precision != 32 && o.precision != 64) return LBM_ERR_INVALID_ARG;
    if (o.top_bc < 0 || o.top_bc > 2 || o.kappa_mode < 0 || o.kappa_mode > 2) return LBM_ERR_INVALID_ARG;
    if (o.hr_sign != 1 && o.hr_sign != -1) return LBM_ERR_INVALID_ARG;
    if (o.h_eval != LBM_H_LOCAL && o.h_eval != LBM_H_LINK_AVG) return LBM_ERR_INVALID_ARG;
    if (o.forcing != LBM_FORCING_EDM && o.forcing != LBM_FORCING_GUO) return LBM_ERR_INVALID_ARG;
    if (o.axis_a_term != LBM_AXIS_A_PRINTED && o.axis_a_term != LBM_AXIS_A_EXPANSION) return LBM_ERR_INVALID_ARG;
    lbm_eos e;
    memset(&e, 0, sizeof(e));
    double T = 0.0, Tc = 0.0;
    if (o.multiphase) {
        if (!eos || (eos->kind != LBM_EOS_VDW && eos->kind != LBM_EOS_CS)) return LBM_ERR_INVALID_ARG;
        e = *eos;
        if (e.kind == LBM_EOS_VDW && !(e.lambda > 0)) return LBM_ERR_INVALID_ARG;
        double rc;
        if (!(e.T_over_Tc > 0) || !lbm::critical_point(e, &Tc, &rc)) return LBM_ERR_INVALID_ARG;
        T = e.T_over_Tc * Tc;
    } else if (eos) {
        e = *eos;
    }
    lbm_axi* h = new (std::nothrow) lbm_axi;
    if (!h) return LBM_ERR_OOM;
    memset(h, 0, sizeof(*h));
    h->nz = nz;
    h->nr = nr;
    h->pitch = pitch_of(nz);
    h->plane = (long long)h->pitch * nr;
    h->precision = o.precision;
    h->tau = tau;
    h->A = A;
    h->eos = e;
    h->T = T;
    h->Tc = Tc;
    h->opts = o;
    h->via_hook = g_alloc != nullptr;
    h->hook_ctx = g_alloc_ctx;
    h->hook_release = g_release;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        (o.precision == 32 ? Ops<float>::prepare() : Ops<double>::prepare()) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LBM_ERR_CUDA;
    }
    const size_t s = o.precision == 32 ? 4 : 8;
    const size_t plane_bytes = (size_t)h->plane * s;
    h->f[0] = dev_alloc(9 * plane_bytes);
    h->f[1] = dev_alloc(9 * plane_bytes);
    h->aux = dev_alloc(4 * plane_bytes);
    h->mout = (double*)dev_alloc(4 * (size_t)nz * nr * sizeof(double));
    h->partial = (double*)dev_alloc(4 * lbm::kReduceBlocks * sizeof(double));
    h->dred = (double*)dev_alloc(4 * sizeof(double));
    h->derr = (int*)dev_alloc(sizeof(int));
    // tile plan of the balanced one-wave step (k_step_single, the batched kernel's single-solve form)
    std::vector<lbm::Tile> tiles;
    std::vector<int> first;
    {
        const int slots = o.precision == 32 ? Ops<float>::batch_resident_ctas(lbm::kStripWide)
                                            : Ops<double>::batch_resident_ctas(lbm::kStripWide);
        int rc = LBM_ERR_CUDA;
        try {
            rc = slots > 0 ? lbm::plan_tiles(&nz, &nr, 1, lbm::kStripWide, slots, tiles, first, nullptr)
                           : LBM_ERR_CUDA;
        } catch (...) {
            rc = LBM_ERR_OOM;
        }
        if (rc != LBM_OK) {
            release_all(h);
            delete h;
            return rc;
        }
    }
    h->ncta = (int)first.size() - 1;
    h->d_tiles = (lbm::Tile*)dev_alloc(tiles.size() * sizeof(lbm::Tile));
    h->d_first = (int*)dev_alloc(first.size() * sizeof(int));
    h->bytes = lbm_axi_footprint(nz, nr, o.precision);
    const bool link = o.h_eval == LBM_H_LINK_AVG && o.axis_terms;
    if (link) {
        h->hb[0] = dev_alloc(3 * plane_bytes);
        h->hb[1] = dev_alloc(3 * plane_bytes);
        h->bytes += 6 * plane_bytes;
    }
    bool ok = h->f[0] && h->f[1] && h->aux && h->mout && h->partial && h->dred && h->derr &&
              h->d_tiles && h->d_first && (!link || (h->hb[0] && h->hb[1]));
    ok = ok && cudaMallocHost(&h->herr, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost(&h->hred, 4 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release_all(h);
        delete h;
        return LBM_ERR_OOM;
    }
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
        h->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            release_all(h);
            delete h;
            return LBM_ERR_CUDA;
        }
        h->own_stream = true;
    }
    h->pf = make_params<float>(h);
    h->pdd = make_params<double>(h);
    h->path = fused_ok(h) ? LBM_PATH_FUSED : LBM_PATH_SPLIT;
    h->rows_per_cta = 0;  // balanced single wave
    if (h->precision == 32) h->pdd = make_params_out(h);
    *h->herr = 0;
    cudaError_t err = cudaSuccess;
    {
        // this solve's tile plan (wide strips, one resident wave)
        err = cudaMemcpy(h->d_tiles, tiles.data(), tiles.size() * sizeof(lbm::Tile), cudaMemcpyHostToDevice);
        if (err == cudaSuccess)
            err = cudaMemcpy(h->d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(h->aux, 0, 4 * plane_bytes, h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (err != cudaSuccess) {
        release_all(h);
        delete h;
        return LBM_ERR_CUDA;
    }
    *out = h;
    return LBM_OK;
}

int lbm_axi_init_device(lbm_axi* h, const double* rho, const double* uz, const double* ur) {
    if (!h || !rho) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaError_t e;
    if (h->precision == 32) {
        e = Ops<float>::init(h->pf, stored_rho_ref(h), rho, uz, ur, (float*)h->f[0], h->stream);
    } else {
        e = Ops<double>::init(h->pdd, stored_rho_ref(h), rho, uz, ur, (double*)h->f[0], h->stream);
    }
    h->cur = 0;
    // a fresh state: clear the sticky error word (the batched kernel skips a solve whose word is set)
    if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    // no arrival halves are pending at the start
    for (int q = 0; q < 2 && e == cudaSuccess && h->hb[0]; q++)
        e = cudaMemsetAsync(h->hb[q], 0, 3 * (size_t)h->plane * (h->precision == 32 ? 4 : 8), h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    h->initialized = true;
    h->pending = LBM_OK;
    return LBM_OK;
}

int lbm_axi_init(lbm_axi* h, const double* rho, const double* uz, const double* ur) {
    if (!h || !rho) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t n = (size_t)h->nz * h->nr;
    double* d_rho = h->mout;
    double* d_uz = uz ? h->mout + n : nullptr;
    double* d_ur = ur ? h->mout + 2 * n : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_rho, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && uz) e = cudaMemcpyAsync(d_uz, uz, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && ur) e = cudaMemcpyAsync(d_ur, ur, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return lbm_axi_init_device(h, d_rho, d_uz, d_ur);
}

int lbm_axi_init_physical_device(lbm_axi* h, const double* rho, const double* uz, const double* ur) {
    int rc = lbm_axi_init_device(h, rho, uz, ur);
    if (rc != LBM_OK) return rc;
    DeviceGuard g(h->device);
    const long long n = (long long)h->nz * h->nr;
    cudaError_t e = enqueue_density(h);
    if (e == cudaSuccess) {
        if (h->precision == 32)
            e = Ops<float>::moments(h->pf, h->pdd, (const float*)h->f[h->cur], (const float*)h->aux, h->mout,
                                    h->stream);
        else
            e = Ops<double>::moments(h->pdd, h->pdd, (const double*)h->f[h->cur], (const double*)h->aux, h->mout,
                                     h->stream);
    }
    if (e == cudaSuccess) {
        k_bare_from_physical<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(n, uz, ur, h->mout + n,
                                                                                   h->mout + 2 * n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    rc = read_error(h);
    if (rc != LBM_OK) return rc;
    return lbm_axi_init_device(h, rho, h->mout + n, h->mout + 2 * n);
}

int lbm_axi_init_physical(lbm_axi* h, const double* rho, const double* uz, const double* ur) {
    if (!h || !rho) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t n = (size_t)h->nz * h->nr;
    double* d = nullptr;
    if (cudaMalloc(&d, 3 * n * sizeof(double)) != cudaSuccess) return LBM_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(d, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && uz) e = cudaMemcpyAsync(d + n, uz, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && ur)
        e = cudaMemcpyAsync(d + 2 * n, ur, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    int rc = e == cudaSuccess ? lbm_axi_init_physical_device(h, d, uz ? d + n : nullptr, ur ? d + 2 * n : nullptr)
                              : LBM_ERR_CUDA;
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    return rc;
}

int lbm_axi_step_async(lbm_axi* h, long long n) {
    if (!h || n < 0) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    if (n == 0) return LBM_OK;
    cudaError_t e = cudaSuccess;
    if (h->cur == 1) {  // graphs start from buffer 0
        e = enqueue_step(h);
        n--;
    }
    const int chunk = chunk_steps(h);
    if (e == cudaSuccess && n >= chunk) {
        if (!h->graph || h->graph_steps != chunk) {
            int rc = build_graph(h, chunk);
            if (rc != LBM_OK) return rc;
        }
        while (n >= chunk && e == cudaSuccess) {
            e = cudaGraphLaunch(h->graph, h->stream);
            n -= chunk;
        }
    }
    while (n > 0 && e == cudaSuccess) {
        e = enqueue_step(h);
        n--;
    }
    if (e != cudaSuccess) {
        h->pending = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int lbm_axi_sync(lbm_axi* h) {
    if (!h) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    int rc = read_error(h);
    if (h->pending != LBM_OK) rc = h->pending;
    h->pending = LBM_OK;
    return rc;
}

int lbm_axi_step(lbm_axi* h, long long n) {
    int rc = lbm_axi_step_async(h, n);
    if (rc != LBM_OK) {
        if (h && rc != LBM_ERR_INVALID_ARG && rc != LBM_ERR_STATE) lbm_axi_sync(h);
        return rc;
    }
    return lbm_axi_sync(h);
}

int lbm_axi_time_kernels(lbm_axi* h, long long n, double* ms) {
    if (!h || n < 0 || !ms) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    cudaEvent_t ev[3];
    for (int q = 0; q < 3; q++) {
        if (cudaEventCreate(&ev[q]) != cudaSuccess) return LBM_ERR_CUDA;
    }
    double acc[2] = {0.0, 0.0};
    cudaError_t e = cudaSuccess;
    for (long long s = 0; s < n && e == cudaSuccess; s++) {
        const int c = h->cur;
        e = cudaEventRecord(ev[0], h->stream);
        if (e == cudaSuccess && h->path == LBM_PATH_SPLIT) e = enqueue_density(h);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
        if (e == cudaSuccess && h->path == LBM_PATH_FUSED) {
            e = enqueue_step(h);
            h->cur = c;
        } else if (e == cudaSuccess) {
            if (h->precision == 32)
                e = Ops<float>::update(h->pf, h->pdd, (const float*)h->f[c], (float*)h->f[c ^ 1],
                                       (const float*)h->aux, h->stream, link_planes<float>(h, c), guo_of(h));
            else
                e = Ops<double>::update(h->pdd, h->pdd, (const double*)h->f[c], (double*)h->f[c ^ 1],
                                        (const double*)h->aux, h->stream, link_planes<double>(h, c), guo_of(h));
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        float t0 = 0.f, t1 = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
        acc[0] += t0;
        acc[1] += t1;
        h->cur = c ^ 1;
    }
    for (int q = 0; q < 3; q++) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    ms[0] = acc[0];
    ms[1] = acc[1];
    return read_error(h);
}

int lbm_axi_moments_device(lbm_axi* h, double* rho, double* uz, double* ur, double* p) {
    if (!h) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    cudaError_t e = enqueue_density(h);
    if (e == cudaSuccess) {
        if (h->precision == 32)
            e = Ops<float>::moments(h->pf, h->pdd, (const float*)h->f[h->cur], (const float*)h->aux, h->mout,
                                    h->stream);
        else
            e = Ops<double>::moments(h->pdd, h->pdd, (const double*)h->f[h->cur], (const double*)h->aux, h->mout,
                                     h->stream);
    }
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    const size_t n = (size_t)h->nz * h->nr;
    double* dst[4] = {rho, uz, ur, p};
    for (int q = 0; q < 4 && e == cudaSuccess; q++) {
        if (dst[q]) e = cudaMemcpyAsync(dst[q], h->mout + q * n, n * sizeof(double), cudaMemcpyDefault, h->stream);
    }
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return read_error(h);
}

int lbm_axi_moments(lbm_axi* h, double* rho, double* uz, double* ur, double* p) {
    return lbm_axi_moments_device(h, rho, uz, ur, p);
}

// ------------------------------------------------------- checkpoint --
// Blob: StateHeader, then the 9 population planes (nr x nz each, z fastest) in
// the storage precision, exactly as the next step will read them.  The header
// records the grid, precision, reference density and every parameter of the
// dynamics, so that a blob only resumes a solve that continues the same run.
namespace {
struct StateHeader {
    char magic[8];  // "LBMAXIS1"
    int32_t version, precision, nz, nr;
    double rho_ref;
    int32_t cur, link_planes, reserved[6];
    // dynamics (format version 2)
    double tau, A, T, T_over_Tc, a, b, R, lambda, g_z;
    int32_t eos_kind, top_bc, axis_terms, multiphase, kappa_mode, hr_sign, h_eval, forcing;
    int32_t axis_a_term, reserved2[5];
};
static_assert(sizeof(StateHeader) == 192, "checkpoint header layout");
const char kStateMagic[8] = {'L', 'B', 'M', 'A', 'X', 'I', 'S', '1'};
constexpr int32_t kStateVersion = 2;

void fill_header(const lbm_axi* h, StateHeader* hd) {
    memset(hd, 0, sizeof(*hd));
    memcpy(hd->magic, kStateMagic, sizeof(kStateMagic));
    hd->version = kStateVersion;
    hd->precision = h->precision;
    hd->nz = h->nz;
    hd->nr = h->nr;
    hd->rho_ref = stored_rho_ref(h);
    hd->cur = h->cur;
    hd->link_planes = h->hb[0] ? 1 : 0;
    hd->tau = h->tau;
    hd->A = h->A;
    hd->T = h->T;
    hd->T_over_Tc = h->opts.multiphase ? h->eos.T_over_Tc : 0.0;
    hd->a = h->opts.multiphase ? h->eos.a : 0.0;
    hd->b = h->opts.multiphase ? h->eos.b : 0.0;
    hd->R = h->opts.multiphase ? h->eos.R : 0.0;
    hd->lambda = h->opts.multiphase ? h->eos.lambda : 0.0;
    hd->g_z = h->opts.g_z;
    hd->eos_kind = h->opts.multiphase ? h->eos.kind : -1;
    hd->top_bc = h->opts.top_bc;
    hd->axis_terms = h->opts.axis_terms ? 1 : 0;
    hd->multiphase = h->opts.multiphase ? 1 : 0;
    hd->kappa_mode = h->opts.kappa_mode;
    hd->hr_sign = h->opts.hr_sign;
    hd->h_eval = h->opts.h_eval;
    hd->forcing = h->opts.forcing;
    hd->axis_a_term = h->opts.axis_a_term;
}

// The blob continues this solve: same layout and the same dynamics, bit for bit.
bool header_matches(const lbm_axi* h, const StateHeader& hd) {
    StateHeader mine;
    fill_header(h, &mine);
    return memcmp(hd.magic, mine.magic, sizeof(mine.magic)) == 0 && hd.version == mine.version &&
           hd.precision == mine.precision && hd.nz == mine.nz && hd.nr == mine.nr && hd.rho_ref == mine.rho_ref &&
           (hd.cur == 0 || hd.cur == 1) && hd.link_planes == mine.link_planes && hd.tau == mine.tau &&
           hd.A == mine.A && hd.T == mine.T && hd.T_over_Tc == mine.T_over_Tc && hd.a == mine.a &&
           hd.b == mine.b && hd.R == mine.R && hd.lambda == mine.lambda && hd.g_z == mine.g_z &&
           hd.eos_kind == mine.eos_kind && hd.top_bc == mine.top_bc && hd.axis_terms == mine.axis_terms &&
           hd.multiphase == mine.multiphase && hd.kappa_mode == mine.kappa_mode && hd.hr_sign == mine.hr_sign &&
           hd.h_eval == mine.h_eval && hd.forcing == mine.forcing && hd.axis_a_term == mine.axis_a_term;
}

// planes in the blob: the 9 populations, then (link-midpoint source) the 3 source planes
int state_planes(const lbm_axi* h) { return h->hb[0] ? 12 : 9; }
size_t state_bytes(const lbm_axi* h) {
    return sizeof(StateHeader) + (size_t)state_planes(h) * h->nz * h->nr * (h->precision == 32 ? 4 : 8);
}
}  // namespace

int lbm_axi_state_bytes(const lbm_axi* h, size_t* bytes) {
    if (!h || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = state_bytes(h);
    return LBM_OK;
}

int lbm_axi_save(lbm_axi* h, void* buf, size_t bytes) {
    if (!h || !buf || bytes < state_bytes(h)) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    StateHeader hd;
    fill_header(h, &hd);
    memcpy(buf, &hd, sizeof(hd));
    const size_t es = h->precision == 32 ? 4 : 8;
    char* dst = static_cast<char*>(buf) + sizeof(hd);
    const char* src = static_cast<const char*>(h->f[h->cur]);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < state_planes(h) && e == cudaSuccess; i++) {
        const char* s = i < 9 ? src + (size_t)i * h->plane * es
                              : static_cast<const char*>(h->hb[h->cur]) + (size_t)(i - 9) * h->plane * es;
        e = cudaMemcpy2DAsync(dst + (size_t)i * h->nz * h->nr * es, h->nz * es, s, (size_t)h->pitch * es,
                              h->nz * es, h->nr, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return read_error(h);
}

int lbm_axi_load(lbm_axi* h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < sizeof(StateHeader)) return LBM_ERR_INVALID_ARG;
    StateHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (!header_matches(h, hd) || bytes < state_bytes(h)) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t es = h->precision == 32 ? 4 : 8;
    const char* src = static_cast<const char*>(buf) + sizeof(hd);
    char* dst = static_cast<char*>(h->f[hd.cur]);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < state_planes(h) && e == cudaSuccess; i++) {
        char* d = i < 9 ? dst + (size_t)i * h->plane * es
                        : static_cast<char*>(h->hb[hd.cur]) + (size_t)(i - 9) * h->plane * es;
        e = cudaMemcpy2DAsync(d, (size_t)h->pitch * es, src + (size_t)i * h->nz * h->nr * es, h->nz * es,
                              h->nz * es, h->nr, cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    h->cur = hd.cur;
    h->initialized = true;
    h->pending = LBM_OK;
    return LBM_OK;
}

int lbm_axi_mass(lbm_axi* h, double* mass_rw, double* mass_plain) {
    if (!h || !mass_rw) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    cudaError_t e = enqueue_density(h);
    if (e == cudaSuccess) {
        if (h->precision == 32)
            e = Ops<float>::mass(h->pf, stored_rho_ref(h), (const float*)h->aux, h->partial, h->dred, h->stream);
        else
            e = Ops<double>::mass(h->pdd, stored_rho_ref(h), (const double*)h->aux, h->partial, h->dred, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hred, h->dred, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    int rc = read_error(h);
    if (rc != LBM_OK) return rc;
    *mass_rw = h->hred[0];
    if (mass_plain) *mass_plain = h->hred[1];
    return LBM_OK;
}

int lbm_axi_pressure_jump(lbm_axi* h, double zc, double rc, double rin, double rout, double* dp) {
    if (!h || !dp || !(rin > 0) || !(rout >= rin)) return LBM_ERR_INVALID_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    DeviceGuard g(h->device);
    cudaError_t e = enqueue_density(h);
    if (e == cudaSuccess) {
        if (h->precision == 32)
            e = Ops<float>::pjump(h->pf, h->pdd, (const float*)h->aux, zc, rc, rin, rout, h->partial, h->dred,
                                  h->stream);
        else
            e = Ops<double>::pjump(h->pdd, h->pdd, (const double*)h->aux, zc, rc, rin, rout, h->partial, h->dred,
                                   h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hred, h->dred, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    int rcode = read_error(h);
    if (rcode != LBM_OK) return rcode;
    if (!(h->hred[1] > 0) || !(h->hred[3] > 0)) return LBM_ERR_INVALID_ARG;
    *dp = h->hred[0] / h->hred[1] - h->hred[2] / h->hred[3];
    return LBM_OK;
}

void lbm_axi_destroy(lbm_axi* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    release_all(h);
    delete h;
}

int lbm_axi_get_tuning(const lbm_axi* h, lbm_axi_tuning* t) {
    if (!h || !t) return LBM_ERR_INVALID_ARG;
    t->path = h->path;
    t->rows_per_cta = h->rows_per_cta;
    return LBM_OK;
}

int lbm_axi_set_tuning(lbm_axi* h, const lbm_axi_tuning* t) {
    if (!h || !t) return LBM_ERR_INVALID_ARG;
    if (t->path != LBM_PATH_FUSED && t->path != LBM_PATH_SPLIT) return LBM_ERR_INVALID_ARG;
    if (t->path == LBM_PATH_FUSED && !fused_ok(h)) return LBM_ERR_INVALID_ARG;
    if (t->path == LBM_PATH_FUSED && fv_of(h) != 0 && t->rows_per_cta != 0) return LBM_ERR_INVALID_ARG;
    if (t->rows_per_cta < 0 || t->rows_per_cta > (1 << 20)) return LBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->path = t->path;
    h->rows_per_cta = t->rows_per_cta;
    return LBM_OK;
}

int lbm_axi_temperature(const lbm_axi* h, double* T, double* Tc) {
    if (!h) return LBM_ERR_INVALID_ARG;
    if (T) *T = h->T;
    if (Tc) *Tc = h->Tc;
    return LBM_OK;
}

int lbm_axi_device_bytes(const lbm_axi* h, size_t* bytes) {
    if (!h || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = h->bytes;
    return LBM_OK;
}

int lbm_eos_critical_temperature(const lbm_eos* eos, double* Tc) {
    if (!eos || !Tc) return LBM_ERR_INVALID_ARG;
    double rc;
    return lbm::critical_point(*eos, Tc, &rc) ? LBM_OK : LBM_ERR_INVALID_ARG;
}

int lbm_eos_coexistence(const lbm_eos* eos, double* rho_v, double* rho_l) {
    if (!eos || !rho_v || !rho_l) return LBM_ERR_INVALID_ARG;
    const double T = lbm::absolute_temperature(*eos);
    if (!(T > 0)) return LBM_ERR_INVALID_ARG;
    return lbm::coexistence(*eos, T, rho_v, rho_l) ? LBM_OK : LBM_ERR_INVALID_ARG;
}

int lbm_eos_pressure(const lbm_eos* eos, double rho, double* p, double* dpdrho) {
    if (!eos || !p) return LBM_ERR_INVALID_ARG;
    const double T = lbm::absolute_temperature(*eos);
    if (!(T > 0)) return LBM_ERR_INVALID_ARG;
    double dp;
    lbm::eos_pressure(*eos, T, rho, p, &dp);
    if (dpdrho) *dpdrho = dp;
    return LBM_OK;
}

int lbm_axi_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return LBM_ERR_INVALID_ARG;
    g_alloc = alloc;
    g_release = release;
    g_alloc_ctx = ctx;
    return LBM_OK;
}

const char* lbm_axi_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_OOM: return "out of memory";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_UNPHYSICAL: return "unphysical state (rho <= 0, psi^2 < 0 or non-finite value)";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
        case LBM_ERR_STATE: return "call out of order (solve not initialised)";
        default: return "unknown error";
    }
}

}  // extern "C"
