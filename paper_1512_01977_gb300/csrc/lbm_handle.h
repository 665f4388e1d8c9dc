// Internal: the solve handle behind the opaque lbm_axi pointer (shared by the
// single-solve API in lbm_axi.cu and the batch API in lbm_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_axi.h"
#include "lbm_device.cuh"
#include "lbm_launch.h"
#include "lbm_tiles.h"

using lbm::Params;

struct lbm_axi {
    int nz, nr, pitch;
    long long plane;
    int precision;
    double tau, A, T, Tc;
    lbm_eos eos;
    lbm_axi_opts opts;
    int device;
    void* f[2];
    int cur;
    void* aux;
    double* mout;     // 4 planes of nz*nr doubles (moments / init staging)
    double* partial;  // reduction partials
    double* dred;     // reduction results (4 doubles)
    int* derr;        // sticky device error word
    int* herr;        // pinned copy
    double* hred;     // pinned reduction results
    cudaStream_t stream;
    bool own_stream;
    bool via_hook;
    void* hook_ctx;
    void (*hook_release)(void*, void*);
    cudaGraphExec_t graph;
    int graph_steps;
    bool initialized;
    int pending;  // error status carried to the next sync
    size_t bytes;
    int path;          // LBM_PATH_FUSED or LBM_PATH_SPLIT
    int rows_per_cta;  // fused path: 0 = balanced wave (k_step_single over the tile plan); > 0 = chunks
                       // (EDM with h_i at the node only)
    lbm::Tile* d_tiles;  // tile plan of this solve alone (wide strips, one resident wave)
    int* d_first;        // [ncta + 1]
    int ncta;
    Params<float> pf;
    Params<double> pdd;
    void* hb[2];  // h at the link midpoint: S0, H_z, H_r planes of the step that wrote f[c] (else null)
};

// Source planes of the link-midpoint reading for a step that reads f[c] (and
// writes f[c^1]); null pointers when the solve evaluates h_i at the node.
template <typename R>
inline lbm::LinkPlanes<R> link_planes(const lbm_axi* h, int c) {
    if (!h->hb[0]) return {nullptr, nullptr};
    return {static_cast<const R*>(h->hb[c]), static_cast<R*>(h->hb[c ^ 1])};
}

// Guo forcing in place of the EDM shift.
inline bool guo_of(const lbm_axi* h) { return h->opts.forcing == LBM_FORCING_GUO; }
// Collision form of the fused kernel (lbm::FV_* bits): Guo forcing, link-midpoint source.
inline int fv_of(const lbm_axi* h) { return (guo_of(h) ? lbm::FV_GUO : 0) | (h->hb[0] ? lbm::FV_LINK : 0); }
// The fused kernel runs this solve: nr >= kStepMinRows, and the Guo and link-source
// forms are compiled with the force and the axis terms on only.
inline bool fused_ok(const lbm_axi* h) {
    return h->nr >= lbm::kStepMinRows && (fv_of(h) == 0 || (h->opts.multiphase && h->opts.axis_terms));
}
// Options the batched engine lacks (such a solve cannot join a batch).
inline bool unbatchable(const lbm_axi* h) { return fv_of(h) != 0; }

// One fused step of this solve over its tile plan (k_step_single, the collision
// form fv_of(h)) reading f[c] and writing f[c^1]; enqueued on h->stream.
cudaError_t lbm_handle_step_tiles(lbm_axi* h, int c);

// Step parity bookkeeping used by the batch API: after n steps run outside
// the handle's own step loop, its current buffer flips when n is odd.
inline void lbm_handle_advance(lbm_axi* h, long long n) {
    if (n & 1) h->cur ^= 1;
}
