// Template bodies of the per-(precision, size) entry points; included by the
// kernels_<prec>_<sizes>.cu units, which instantiate Sized<T, SZ> for a few
// sizes each.
#pragma once
#include "pipeline.cuh"
#include "rows_tm.cuh"
#include <algorithm>
#include <type_traits>

namespace cmif {

// Sizes with the 16-lane variant of the column transforms (FP32 only).
template <typename T, int SZ>
constexpr bool kHasColVariant = std::is_same<T, float>::value && SZ >= 1024 && is_pow2(SZ);

// Opt the kernel in to `bytes` of dynamic shared memory.  Without the attribute,
// static plus dynamic shared memory must stay within 48 KB, so a kernel with a
// little static memory (a work index, an abort flag) fails to launch just below
// 48 KB of dynamic memory: set it from 32 KB up.
template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
    if (bytes <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int Q>
static cudaError_t launch_fwd_rows(const int32_t* X, const uint8_t* MX, const double* WX, int H, int W, int K, int Qs,
                                   cpx<T>* T1, const Tw<T>& tw, DevStatus* st, int conditional, int* popc,
                                   const unsigned char* need, cudaStream_t s) {
    using C = FwdRowsCfg<T, Q>;
    auto kern = k_fwd_rows<T, Q>;
    cudaError_t e = ensure_smem(kern, C::smem(Q, true));
    if (e != cudaSuccess) return e;
    dim3 grid(H, ((K + 1) / 2 + C::TPB - 1) / C::TPB);
    kern<<<grid, C::THREADS, C::smem(W, WX != nullptr), s>>>(X, MX, WX, H, W, K, Qs, T1, tw, st, conditional, popc,
                                                             need);
    return cudaGetLastError();
}

template <typename T, int P, int MMAX>
static cudaError_t launch_fwd_cols(const cpx<T>* T1, int H, int K, int Qh, int Qs, cpx<T>* F, const Tw<T>& tw,
                                   const DevStatus* st, int conditional, T out_scale, const unsigned char* need,
                                   int slices, cudaStream_t s) {
    using C = ColCfg<T, P, MMAX>;
    auto kern = k_fwd_cols<T, P, MMAX>;
    cudaError_t e = ensure_smem(kern, C::smem(P));
    if (e != cudaSuccess) return e;
    dim3 grid((Qh + C::TPB - 1) / C::TPB, K);
    kern<<<grid, C::THREADS, C::smem(H), s>>>(T1, H, K, Qh, Qs, F, tw, st, conditional, out_scale, need, slices);
    return cudaGetLastError();
}

template <typename T, int P, bool VOL, int MMAX>
static cudaError_t launch_pair_cols(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    using C = PairColsCfg<T, P, MMAX>;
    auto kern = k_pair_cols<T, P, VOL, MMAX>;
    const size_t smem = pair_cols_smem<T, P, MMAX>();
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    // persistent grid: every resident block slot of the device, at most one per item
    static int per_sm = -1;
    if (per_sm < 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::THREADS, smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    const long long np = a.plist ? a.chunk_cap : (long long)g.KA * g.KB;  // list mode: at most chunk_cap pairs
    const long long items = np * ((g.Qh + C::TPB - 1) / C::TPB) * (VOL ? g.Dz : g.units);
    const int bps = a.cols_bps > 0 && a.cols_bps < per_sm ? a.cols_bps : per_sm;
    const long long slots = a.num_sms > 0 ? (long long)bps * a.num_sms : items;
    const int grid = (int)(items < slots ? items : slots);
    e = cudaMemsetAsync(a.work_ctr, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    kern<<<grid, C::THREADS, smem, s>>>(a.FA, a.FB, g.KA, g.KB, g.Qh, g.HA, g.HB, g.R, g.Qs, g.r0, g.r1, a.Y, a.tw,
                                        a.st, a.conditional, a.work_ctr, g.DA, g.DB, g.R2, a.plist, a.lrange,
                                        a.chunk_off, a.chunk_cap, VOL ? 1 : g.units);
    return cudaGetLastError();
}

template <typename T, int Q, bool NMI>
static cudaError_t launch_pair_rows_v(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    using C = RowCfg<T, Q>;
    if constexpr (sizeof(T) == 4 && (Q == 512 || Q == 1024 || Q == 2048)) {
        if (a.tm_cols > 0 && !a.counts) {  // debug count maps: the generic kernel below
            const bool ext = a.ov_slot || a.pair_res || a.conditional || a.wait_polls > 0 || a.withhold_row >= 0;
            // the multi-unit kernel lives in its own translation unit (kernels_f32_rows_units.cu):
            // compiled next to the plain one, it changed the plain kernel's register allocation
            if (!ext && g.units > 1) return launch_rows_tm_units<Q, NMI>(g, a, s);
            auto kern = ext ? k_pair_rows_tm<Q, NMI, 2> : k_pair_rows_tm<Q, NMI, 0>;
            cudaError_t e = ensure_smem(kern, RowTmCfg<Q>::SMEM);
            if (e != cudaSuccess) return e;
            kern<<<a.rows_grid, RowTmCfg<Q>::THREADS, RowTmCfg<Q>::SMEM, s>>>(
                a.Y, g, a.tw, a.mi, a.n, a.st, a.tm_cols, a.wait_polls > 0 ? a.wait_polls : kDefaultWaitPolls,
                a.withhold_row, a.conditional, a.ov, a.ov_slot, a.pair_res);
            return cudaGetLastError();
        }
    }
    const size_t smem = pair_rows_smem<T, Q>(g.KB, a.cb_smem);
    if (a.cb_smem) {
        auto kern = k_pair_rows<T, Q, true, NMI>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<a.rows_grid, C::THREADS, smem, s>>>(a.Y, g, a.tw, a.cb_global, a.mi, a.n, a.counts, a.st,
                                                   a.prec_slot, a.conditional, a.ov, a.ov_slot, a.pair_res);
    } else if constexpr (Q > 512) {  // Q <= 512: K_B (<= 64) x Q floats always fit in shared memory
        auto kern = k_pair_rows<T, Q, false, NMI>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<a.rows_grid, C::THREADS, smem, s>>>(a.Y, g, a.tw, a.cb_global, a.mi, a.n, a.counts, a.st,
                                                   a.prec_slot, a.conditional, a.ov, a.ov_slot, a.pair_res);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// MI or NMI epilogue (CMIF_FLAG_NMI)
template <typename T, int Q>
static cudaError_t launch_pair_rows(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    return a.nmi ? launch_pair_rows_v<T, Q, true>(g, a, s) : launch_pair_rows_v<T, Q, false>(g, a, s);
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::fwd_rows(const Geom& g, const PipeArgs<T>& a, bool b_side, cudaStream_t s) {
    const double* wb = a.weighted ? a.WB : nullptr;
    const double* wa = a.weighted ? a.WA : nullptr;
    // volumes: the D slices of H rows are D * H rows of one image
    return b_side ? launch_fwd_rows<T, SZ>(a.B, a.MB, wb, g.DB * g.HB, g.WB, g.KB, g.Qs, a.T1B, a.tw, a.st,
                                           a.conditional, a.popB, a.needB, s)
                  : launch_fwd_rows<T, SZ>(a.A, a.MA, wa, g.DA * g.HA, g.WA, g.KA, g.Qs, a.T1A, a.tw, a.st,
                                           a.conditional, a.popA, a.needA, s);
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::fwd_cols(const Geom& g, const PipeArgs<T>& a, bool b_side, cudaStream_t s) {
    // B's spectra carry the 1/(P Q) of the unnormalised inverse transform (a power of two: exact)
    // volumes: K * D slice planes of H rows each (plane index label * D + z)
    auto go = [&](auto mm) {
        constexpr int MM = decltype(mm)::value;
        return b_side ? launch_fwd_cols<T, SZ, MM>(a.T1B, g.HB, g.KB * g.DB, g.Qh, g.Qs, a.FB, a.tw, a.st,
                                                   a.conditional, T(1.0 / ((double)g.P * (double)g.Q)), a.needB,
                                                   g.DB, s)
                      : launch_fwd_cols<T, SZ, MM>(a.T1A, g.HA, g.KA * g.DA, g.Qh, g.Qs, a.FA, a.tw, a.st,
                                                   a.conditional, T(1), a.needA, g.DA, s);
    };
    if constexpr (kHasColVariant<T, SZ>) {
        if (a.col_m == 16) return go(std::integral_constant<int, 16>{});
    }
    return go(std::integral_constant<int, max_m<T>()>{});
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::pair_cols(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    if constexpr (kHasColVariant<T, SZ>) {
        if (a.col_m == 16)
            return g.Dz > 1 ? launch_pair_cols<T, SZ, true, 16>(g, a, s) : launch_pair_cols<T, SZ, false, 16>(g, a, s);
    }
    constexpr int MM = max_m<T>();
    return g.Dz > 1 ? launch_pair_cols<T, SZ, true, MM>(g, a, s) : launch_pair_cols<T, SZ, false, MM>(g, a, s);
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::pair_rows(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    return launch_pair_rows<T, SZ>(g, a, s);
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::pair_rows_counts(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    using C = RowCntCfg<T, SZ>;
    auto kern = k_pair_rows_counts<T, SZ>;
    cudaError_t e = ensure_smem(kern, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long tasks = (long long)a.chunk_cap * (g.r1 - g.r0);
    const long long blocks = std::min<long long>((tasks + C::NT - 1) / C::NT, 8LL * (a.num_sms > 0 ? a.num_sms : 152));
    kern<<<(int)std::max<long long>(1, blocks), C::THREADS, C::SMEM, s>>>(a.Y, g, a.tw, a.lrange, a.chunk_off,
                                                                          a.chunk_cap, a.ov, a.st);
    return cudaGetLastError();
}

template <typename T, int SZ>
size_t Sized<T, SZ>::rows_smem(int KB, bool cb_smem) {
    return pair_rows_smem<T, SZ>(KB, cb_smem);
}

template <typename T, int SZ>
int Sized<T, SZ>::rows_threads() {
    return RowCfg<T, SZ>::THREADS;
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::rows_max_blocks(int KB, bool cb_smem, int* out) {
    const size_t smem = pair_rows_smem<T, SZ>(KB, cb_smem);
    if (cb_smem) {
        auto kern = k_pair_rows<T, SZ, true, false>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, RowCfg<T, SZ>::THREADS, smem);
    }
    if constexpr (SZ > 512) {
        auto kern = k_pair_rows<T, SZ, false, false>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, RowCfg<T, SZ>::THREADS, smem);
    } else {
        return cudaErrorInvalidValue;  // not reached: the B-marginals always fit in shared memory
    }
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::pair_rows_w(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    if constexpr (std::is_same<T, double>::value) {
        using C = RowWCfg<SZ>;
        cudaError_t e = ensure_smem(k_pair_rows_w<SZ>, C::SMEM);
        if (e != cudaSuccess) return e;
        k_pair_rows_w<SZ><<<a.rows_grid_w, C::THREADS, C::SMEM, s>>>(a.Y, g, a.tw, a.cbw, a.mi, a.nw, a.st);
        return cudaGetLastError();
    } else {
        (void)g; (void)a; (void)s;
        return cudaErrorNotSupported;  // weighted maps need FP64 transforms
    }
}

template <typename T, int SZ>
size_t Sized<T, SZ>::rows_w_smem() {
    if constexpr (std::is_same<T, double>::value) return RowWCfg<SZ>::SMEM;
    else return 0;
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::rows_w_max_blocks(int* out) {
    if constexpr (std::is_same<T, double>::value) {
        using C = RowWCfg<SZ>;
        cudaError_t e = ensure_smem(k_pair_rows_w<SZ>, C::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pair_rows_w<SZ>, C::THREADS, C::SMEM);
    } else {
        *out = 0;
        return cudaSuccess;
    }
}

template <typename T, int SZ>
int Sized<T, SZ>::tm_cols(int KB) {
    if constexpr (sizeof(T) == 4 && (SZ == 512 || SZ == 1024 || SZ == 2048)) {
        const int need = tm_cols_needed(KB, RowTmCfg<SZ>::U);
        return need <= 512 ? tm_alloc_cols(need) : 0;
    } else {
        (void)KB;
        return 0;
    }
}

template <typename T, int SZ>
cudaError_t Sized<T, SZ>::tm_max_blocks(int* out) {
    if constexpr (sizeof(T) == 4 && (SZ == 512 || SZ == 1024 || SZ == 2048)) {
        cudaError_t e = ensure_smem(k_pair_rows_tm<SZ, false, 0>, RowTmCfg<SZ>::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pair_rows_tm<SZ, false, 0>, RowTmCfg<SZ>::THREADS,
                                                             RowTmCfg<SZ>::SMEM);
    } else {
        *out = 0;
        return cudaSuccess;
    }
}

}  // namespace cmif
