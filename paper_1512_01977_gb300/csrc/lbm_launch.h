// Host-side launchers of the kernels, one explicit instantiation per
// precision (kernels_f32.cu, kernels_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_tiles.h"

namespace lbm {

constexpr int kReduceBlocks = 304;  // 2 x 152 SMs; fixed so reductions are reproducible
constexpr int kStepMinRows = 16;    // the single-pass kernel needs single reflections at the walls
// z-columns per CTA of the two compiled forms of the batched kernel (the wide
// one is the default; the autotuner may pick the narrow one for small grids).
// 112: with 128 threads of two columns each, stages L, D, U and C fill 124,
// 120, 116 and 112 of them, and strip origins stay 64-byte aligned; measured
// fastest of the even widths 96 ... 116 on the 4096 x 2048 wave.
constexpr int kStripNarrow = 64, kStripWide = 112;

template <typename R>
struct Ops {
    // kernel (a): gather, rho/j, psi; raises bits in *err.
    // lk: the link-midpoint source planes (null: h_i at the node).
    static cudaError_t density(const Params<R>& p, const R* f, R* aux, int* err, cudaStream_t s,
                               LinkPlanes<R> lk = {nullptr, nullptr});
    // kernel (b): the fused stream + force + EDM + axisymmetric source + collide step
    // (guo: Guo forcing in place of the EDM shift).
    static cudaError_t update(const Params<R>& p, const Params<double>& pd, const R* f, R* fout, const R* aux,
                              cudaStream_t s, LinkPlanes<R> lk = {nullptr, nullptr}, bool guo = false);
    // rho, physical u, P_k of the current state into mout[4][nz*nr] (after density()).
    static cudaError_t moments(const Params<R>& p, const Params<double>& pd, const R* f, const R* aux,
                               double* mout, cudaStream_t s);
    static cudaError_t init(const Params<R>& p, double rho_ref, const double* rho, const double* uz,
                            const double* ur, R* f, cudaStream_t s);
    // kernel (c): out[0] = sum (j+1/2) rho, out[1] = sum rho.
    static cudaError_t mass(const Params<R>& p, double rho_ref, const R* aux, double* partial, double* out,
                            cudaStream_t s);
    // out[0..3] = sum P_k inside, count inside, sum P_k outside, count outside.
    static cudaError_t pjump(const Params<R>& p, const Params<double>& pd, const R* aux, double zc, double rc,
                             double rin, double rout, double* partial, double* out, cudaStream_t s);
    // dynamic shared memory of one k_update CTA, bytes
    static size_t update_smem();
    // one-time kernel attributes (shared-memory opt-in); call outside stream capture
    static cudaError_t prepare();
    // kernel (b'): the whole step in one pass (needs nr >= kStepMinRows); rows_per_cta
    // rows of each z-strip per CTA.
    static cudaError_t step(const Params<R>& p, const R* f, R* fout, int rows_per_cta, int* err, cudaStream_t s);
    static size_t step_smem();
    static int step_strip();  // z-columns per CTA of the single-pass kernel
    // Batched fused step: ncta CTAs, CTA c marching tiles first[c] .. first[c + 1] - 1
    // (device arrays planned by plan_tiles for this strip width); strip: kStripNarrow
    // or kStripWide z-columns per CTA.  fv: FV_* collision form, nonzero only with
    // kStripWide and mp && ax (cudaErrorInvalidValue otherwise).
    static cudaError_t step_batch(const BatchSolve<R>* solves, const Tile* tiles, const int* first, int ncta,
                                  bool mp, bool ax, int parity, int strip, int* err, cudaStream_t s, int fv = 0);
    // The fused step of one solve, descriptor by value (kStripWide tiles; same
    // arithmetic as step_batch with a batch of one).
    static cudaError_t step_single(const BatchSolve<R>& solve, const Tile* tiles, const int* first, int ncta,
                                   bool mp, bool ax, int parity, int* err, cudaStream_t s, int fv = 0);
    // The batched step with the descriptors as one kernel argument (FP32; n <=
    // BatchTable<R>::N solves; cudaErrorNotSupported in FP64).
    static cudaError_t step_table(const BatchTable<R>& table, const Tile* tiles, const int* first, int ncta,
                                  bool mp, bool ax, int parity, int strip, int* err, cudaStream_t s);
    static int batch_resident_ctas(int strip);
    static size_t batch_smem(int strip);
};

}  // namespace lbm
