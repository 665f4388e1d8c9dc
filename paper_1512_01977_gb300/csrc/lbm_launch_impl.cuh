// Definitions of Ops<R>; included once per precision.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

// Tile of kernel (b) per precision: TZ nodes along z (coalesced) x TR rows.
template <typename R>
struct UpdateTile;
template <>
struct UpdateTile<float> {
    // 32 x 32: 512 us per launch through the C ABI on the 4096 x 2048 wave against
    // 559 us for 32 x 16 (less halo work); wider tiles lose occupancy (64 x 16: +19 %)
    static constexpr int TZ = 32, TR = 32;
};
template <>
struct UpdateTile<double> {
    static constexpr int TZ = 32, TR = 8;
};

template <typename R>
size_t Ops<R>::update_smem() {
    using T = UpdateTile<R>;
    return sizeof(R) * (size_t)TileShape<T::TZ, T::TR>::elems;
}

template <typename R>
static cudaError_t launch_update(const Params<R>& p, const Params<double>& pd, const R* f, R* fout, const R* aux,
                                 double* mout, bool moments, cudaStream_t s, LinkPlanes<R> lk, bool guo) {
    using T = UpdateTile<R>;
    const size_t smem = Ops<R>::update_smem();
    dim3 grid((p.nz + T::TZ - 1) / T::TZ, (p.nr + T::TR - 1) / T::TR);
    if (moments) {
        k_update<R, T::TZ, T::TR, true><<<grid, 256, smem, s>>>(p, pd, f, nullptr, aux, mout, lk);
    } else if (guo) {
        k_update<R, T::TZ, T::TR, false, true><<<grid, 256, smem, s>>>(p, pd, f, fout, aux, nullptr, lk);
    } else {
        k_update<R, T::TZ, T::TR, false><<<grid, 256, smem, s>>>(p, pd, f, fout, aux, nullptr, lk);
    }
    return cudaGetLastError();
}

// Strip width and rows per iteration of the fused kernel per precision.
template <typename R>
struct StepTile;
// CP: columns per thread (2: march2, pairs of nodes with packed FP32 arithmetic).
template <>
struct StepTile<float> {
    static constexpr int TZ = 112, RR = 2, CP = 2, MINB = 4;  // 128 threads, 45.3 KB of rings
};
template <>
struct StepTile<double> {
    static constexpr int TZ = 64, RR = 2, CP = 1, MINB = 2;  // 160 threads, 71.7 KB of rings
};

template <typename R>
size_t Ops<R>::step_smem() {
    return sizeof(R) * (size_t)StepShape<StepTile<R>::TZ, StepTile<R>::RR>::elems;
}

template <typename R>
int Ops<R>::step_strip() {
    return StepTile<R>::TZ;
}

// The four compiled forms of the fused kernel (force on/off x axis terms on/off).
template <typename R, bool MP, bool AX>
static auto step_kernel() {
    return k_step<R, StepTile<R>::TZ, StepTile<R>::RR, StepTile<R>::CP, StepTile<R>::MINB, MP, AX>;
}

template <typename R>
static cudaError_t set_step_attr(int smem) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<R, true, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_kernel<R, true, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_kernel<R, false, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_kernel<R, false, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <typename R>
static cudaError_t single_prepare();
template <typename R, int TZ>
static cudaError_t table_prepare();

template <typename R>
cudaError_t Ops<R>::prepare() {
    using T = UpdateTile<R>;
    const int smem = (int)update_smem();
    cudaError_t e = cudaFuncSetAttribute(k_update<R, T::TZ, T::TR, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_update<R, T::TZ, T::TR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_update<R, T::TZ, T::TR, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = set_step_attr<R>((int)step_smem());
    // the batched kernel (also the default single-solve step): attributes and
    // occupancy are settled here, outside any stream capture
    if (e == cudaSuccess && (batch_resident_ctas(kStripNarrow) <= 0 || batch_resident_ctas(kStripWide) <= 0))
        e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = single_prepare<R>();  // the single-solve form of the fused kernel
    if constexpr (sizeof(R) == 4) {  // the argument-table form of the batched kernel
        if (e == cudaSuccess) e = table_prepare<R, kStripNarrow>();
        if (e == cudaSuccess) e = table_prepare<R, kStripWide>();
    }
    return e;
}

// CTAs of the fused kernel that fit on the device at once (one wave).
template <typename R>
static int step_resident_ctas() {
    static int cached = 0;
    if (cached > 0) return cached;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<R, true, true>(),
                                                      StepShape<StepTile<R>::TZ, StepTile<R>::RR, StepTile<R>::CP>::NT,
                                                      Ops<R>::step_smem()) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    cached = sms * per_sm;
    return cached;
}

template <typename R>
cudaError_t Ops<R>::step(const Params<R>& p, const R* f, R* fout, int rows_per_cta, int* err, cudaStream_t s) {
    constexpr int TZ = StepTile<R>::TZ, RR = StepTile<R>::RR, CP = StepTile<R>::CP;
    constexpr int NT = StepShape<TZ, RR, CP>::NT;
    dim3 grid;
    if (rows_per_cta > 0) {
        grid = dim3((p.nz + TZ - 1) / TZ, (p.nr + rows_per_cta - 1) / rows_per_cta);
    } else {
        // balanced single wave; no CTA gets less than 16 rows of work
        const long long total = (long long)((p.nz + TZ - 1) / TZ) * p.nr;
        long long n = step_resident_ctas<R>();
        if (n > (total + 15) / 16) n = (total + 15) / 16;
        grid = dim3((unsigned)(n > 0 ? n : 1));
    }
    const size_t smem = step_smem();
    if (p.multiphase && p.axis)
        step_kernel<R, true, true>()<<<grid, NT, smem, s>>>(p, f, fout, rows_per_cta, err);
    else if (p.multiphase)
        step_kernel<R, true, false>()<<<grid, NT, smem, s>>>(p, f, fout, rows_per_cta, err);
    else if (p.axis)
        step_kernel<R, false, true>()<<<grid, NT, smem, s>>>(p, f, fout, rows_per_cta, err);
    else
        step_kernel<R, false, false>()<<<grid, NT, smem, s>>>(p, f, fout, rows_per_cta, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::density(const Params<R>& p, const R* f, R* aux, int* err, cudaStream_t s, LinkPlanes<R> lk) {
    dim3 block(32, 8), grid((p.nz + 31) / 32, (p.nr + 7) / 8);
    k_density<R><<<grid, block, 0, s>>>(p, f, aux, err, lk);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::update(const Params<R>& p, const Params<double>& pd, const R* f, R* fout, const R* aux,
                           cudaStream_t s, LinkPlanes<R> lk, bool guo) {
    return launch_update<R>(p, pd, f, fout, aux, nullptr, false, s, lk, guo);
}

template <typename R>
cudaError_t Ops<R>::moments(const Params<R>& p, const Params<double>& pd, const R* f, const R* aux, double* mout,
                            cudaStream_t s) {
    return launch_update<R>(p, pd, f, nullptr, aux, mout, true, s, LinkPlanes<R>{nullptr, nullptr}, false);
}

template <typename R>
cudaError_t Ops<R>::init(const Params<R>& p, double rho_ref, const double* rho, const double* uz, const double* ur,
                         R* f, cudaStream_t s) {
    dim3 block(32, 8), grid((p.nz + 31) / 32, (p.nr + 7) / 8);
    k_init<R><<<grid, block, 0, s>>>(p, rho_ref, rho, uz, ur, f);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::mass(const Params<R>& p, double rho_ref, const R* aux, double* partial, double* out,
                         cudaStream_t s) {
    k_mass<R><<<kReduceBlocks, 256, 0, s>>>(p, rho_ref, aux, partial);
    k_reduce_final<2><<<1, 32, 0, s>>>(partial, kReduceBlocks, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::pjump(const Params<R>& p, const Params<double>& pd, const R* aux, double zc, double rc,
                          double rin, double rout, double* partial, double* out, cudaStream_t s) {
    k_pjump<R><<<kReduceBlocks, 256, 0, s>>>(p, pd, aux, zc, rc, rin, rout, partial);
    k_reduce_final<4><<<1, 32, 0, s>>>(partial, kReduceBlocks, out);
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

// Batched kernel forms: strip width kStripNarrow or kStripWide (the autotuner picks), force and
// axis terms compiled in or out.
// Resident CTAs per SM the launch bounds ask for: what shared memory allows at
// each width (FP32 two columns per thread: 45.3 KB / 26.9 KB of rings; FP64
// one column: 90.6 KB / 53.8 KB).
template <typename R, int TZ>
struct BatchMinBlocks {
    static constexpr int value = sizeof(R) == 4 ? (TZ == kStripWide ? 4 : 5) : (TZ == kStripWide ? 2 : 3);
};

template <typename R, int TZ>
struct BatchTile {
    static constexpr int RR = 2;
    static constexpr int CP = StepTile<R>::CP;
    static constexpr int MINB = BatchMinBlocks<R, TZ>::value;
    static constexpr int NT = StepShape<TZ, RR, CP>::NT;
    static size_t smem() { return sizeof(R) * (size_t)StepShape<TZ, RR, CP>::elems; }
};

template <typename R, int TZ, bool MP, bool AX, int FV = 0>
static auto batch_kernel() {
    return k_step_batch<R, TZ, BatchTile<R, TZ>::RR, BatchTile<R, TZ>::CP, BatchTile<R, TZ>::MINB, MP, AX, FV>;
}

template <typename R, bool MP, bool AX, int FV = 0>
static auto single_kernel() {
    constexpr int TZ = kStripWide;
    return k_step_single<R, TZ, BatchTile<R, TZ>::RR, BatchTile<R, TZ>::CP, BatchTile<R, TZ>::MINB, MP, AX, FV>;
}

template <typename R>
static cudaError_t single_prepare() {
    const int smem = (int)BatchTile<R, kStripWide>::smem();
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(single_kernel<R, true, true>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, true, false>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, false, true>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, false, false>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, true, true, FV_GUO>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, true, true, FV_LINK>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(single_kernel<R, true, true, FV_GUO | FV_LINK>(), a, smem);
    return e;
}

template <typename R, int TZ>
static cudaError_t batch_prepare() {
    const int smem = (int)BatchTile<R, TZ>::smem();
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<R, TZ, true, true>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<R, TZ, true, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<R, TZ, false, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<R, TZ, false, false>(),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (TZ == kStripWide) {  // the collision variants (Guo, link source): wide strips, force + axis
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_kernel<R, TZ, true, true, FV_GUO>(),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_kernel<R, TZ, true, true, FV_LINK>(),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_kernel<R, TZ, true, true, FV_GUO | FV_LINK>(),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return e;
}

template <typename R, int TZ, bool MP, bool AX>
static auto table_kernel() {
    return k_step_table<R, TZ, BatchTile<R, TZ>::RR, BatchTile<R, TZ>::CP, BatchTile<R, TZ>::MINB, MP, AX>;
}

template <typename R, int TZ>
static cudaError_t table_prepare() {
    const int smem = (int)BatchTile<R, TZ>::smem();
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(table_kernel<R, TZ, true, true>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(table_kernel<R, TZ, true, false>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(table_kernel<R, TZ, false, true>(), a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(table_kernel<R, TZ, false, false>(), a, smem);
    return e;
}

template <typename R, int TZ>
static cudaError_t launch_table(const BatchTable<R>& table, const Tile* tiles, const int* first, int ncta, bool mp,
                                bool ax, int parity, int* err, cudaStream_t s) {
    using T = BatchTile<R, TZ>;
    const size_t smem = T::smem();
    if (mp && ax)
        table_kernel<R, TZ, true, true>()<<<ncta, T::NT, smem, s>>>(table, tiles, first, parity, err);
    else if (mp)
        table_kernel<R, TZ, true, false>()<<<ncta, T::NT, smem, s>>>(table, tiles, first, parity, err);
    else if (ax)
        table_kernel<R, TZ, false, true>()<<<ncta, T::NT, smem, s>>>(table, tiles, first, parity, err);
    else
        table_kernel<R, TZ, false, false>()<<<ncta, T::NT, smem, s>>>(table, tiles, first, parity, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::step_table(const BatchTable<R>& table, const Tile* tiles, const int* first, int ncta, bool mp,
                               bool ax, int parity, int strip, int* err, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        if (ncta <= 0) return cudaErrorInvalidConfiguration;
        return strip == kStripNarrow
                   ? launch_table<R, kStripNarrow>(table, tiles, first, ncta, mp, ax, parity, err, s)
                   : launch_table<R, kStripWide>(table, tiles, first, ncta, mp, ax, parity, err, s);
    } else {
        return cudaErrorNotSupported;
    }
}

template <typename R>
size_t Ops<R>::batch_smem(int strip) {
    return strip == kStripNarrow ? BatchTile<R, kStripNarrow>::smem() : BatchTile<R, kStripWide>::smem();
}

template <typename R>
int Ops<R>::batch_resident_ctas(int strip) {
    static int cached[2] = {0, 0};
    const int slot = strip == kStripNarrow ? 0 : 1;
    if (cached[slot] > 0) return cached[slot];
    if ((strip == kStripNarrow ? batch_prepare<R, kStripNarrow>() : batch_prepare<R, kStripWide>()) != cudaSuccess) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    cudaError_t e = strip == kStripNarrow ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                      &per_sm, batch_kernel<R, kStripNarrow, true, true>(), BatchTile<R, kStripNarrow>::NT,
                                      BatchTile<R, kStripNarrow>::smem())
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                      &per_sm, batch_kernel<R, kStripWide, true, true>(), BatchTile<R, kStripWide>::NT,
                                      BatchTile<R, kStripWide>::smem());
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    cached[slot] = sms * per_sm;
    return cached[slot];
}

template <typename R, int TZ>
static cudaError_t launch_batch(const BatchSolve<R>* solves, const Tile* tiles, const int* first, int ncta, bool mp,
                                bool ax, int fv, int parity, int* err, cudaStream_t s) {
    using T = BatchTile<R, TZ>;
    const size_t smem = T::smem();
    if (fv != 0) {
        if constexpr (TZ == kStripWide) {
            if (!(mp && ax)) return cudaErrorInvalidValue;
            if (fv == FV_GUO)
                batch_kernel<R, TZ, true, true, FV_GUO>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
            else if (fv == FV_LINK)
                batch_kernel<R, TZ, true, true, FV_LINK>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
            else if (fv == (FV_GUO | FV_LINK))
                batch_kernel<R, TZ, true, true, FV_GUO | FV_LINK>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first,
                                                                                           parity, err);
            else
                return cudaErrorInvalidValue;
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (mp && ax)
        batch_kernel<R, TZ, true, true>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
    else if (mp)
        batch_kernel<R, TZ, true, false>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
    else if (ax)
        batch_kernel<R, TZ, false, true>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
    else
        batch_kernel<R, TZ, false, false>()<<<ncta, T::NT, smem, s>>>(solves, tiles, first, parity, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::step_single(const BatchSolve<R>& solve, const Tile* tiles, const int* first, int ncta, bool mp,
                                bool ax, int parity, int* err, cudaStream_t s, int fv) {
    using T = BatchTile<R, kStripWide>;
    if (ncta <= 0) return cudaErrorInvalidConfiguration;
    const size_t smem = T::smem();
    if (fv != 0 && !(mp && ax)) return cudaErrorInvalidValue;
    if (fv == FV_GUO)
        single_kernel<R, true, true, FV_GUO>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else if (fv == FV_LINK)
        single_kernel<R, true, true, FV_LINK>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else if (fv == (FV_GUO | FV_LINK))
        single_kernel<R, true, true, FV_GUO | FV_LINK>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else if (fv != 0)
        return cudaErrorInvalidValue;
    else if (mp && ax)
        single_kernel<R, true, true>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else if (mp)
        single_kernel<R, true, false>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else if (ax)
        single_kernel<R, false, true>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    else
        single_kernel<R, false, false>()<<<ncta, T::NT, smem, s>>>(solve, tiles, first, parity, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Ops<R>::step_batch(const BatchSolve<R>* solves, const Tile* tiles, const int* first, int ncta, bool mp,
                               bool ax, int parity, int strip, int* err, cudaStream_t s, int fv) {
    if (ncta <= 0) return cudaErrorInvalidConfiguration;
    return strip == kStripNarrow
               ? launch_batch<R, kStripNarrow>(solves, tiles, first, ncta, mp, ax, fv, parity, err, s)
               : launch_batch<R, kStripWide>(solves, tiles, first, ncta, mp, ax, fv, parity, err, s);
}

}  // namespace lbm
