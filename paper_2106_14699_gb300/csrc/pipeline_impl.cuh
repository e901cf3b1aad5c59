// Template bodies of the launch sequence; included by kernels_f32.cu and
// kernels_f64.cu, which instantiate them for one precision each.
#pragma once
#include "pipeline.cuh"
#include "rows_tm.cuh"
#include <type_traits>

namespace cmif {

template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define CMIF_SIZE_SWITCH(N, ...)              \
    switch (N) {                               \
        case 16: { constexpr int SZ = 16; __VA_ARGS__; } break;     \
        case 32: { constexpr int SZ = 32; __VA_ARGS__; } break;     \
        case 64: { constexpr int SZ = 64; __VA_ARGS__; } break;     \
        case 128: { constexpr int SZ = 128; __VA_ARGS__; } break;   \
        case 256: { constexpr int SZ = 256; __VA_ARGS__; } break;   \
        case 512: { constexpr int SZ = 512; __VA_ARGS__; } break;   \
        case 1024: { constexpr int SZ = 1024; __VA_ARGS__; } break; \
        case 2048: { constexpr int SZ = 2048; __VA_ARGS__; } break; \
        case 4096: { constexpr int SZ = 4096; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;               \
    }

template <typename T, int Q>
static cudaError_t launch_fwd_rows(const int32_t* X, const uint8_t* MX, int H, int W, int K, int Qs, cpx<T>* T1,
                                   const Tw<T>& tw, DevStatus* st, int conditional, cudaStream_t s) {
    using C = FwdRowsCfg<T, Q>;
    auto kern = k_fwd_rows<T, Q>;
    cudaError_t e = ensure_smem(kern, C::smem(Q));
    if (e != cudaSuccess) return e;
    dim3 grid(H, ((K + 1) / 2 + C::TPB - 1) / C::TPB);
    kern<<<grid, C::THREADS, C::smem(W), s>>>(X, MX, H, W, K, Qs, T1, tw, st, conditional);
    return cudaGetLastError();
}

template <typename T, int P>
static cudaError_t launch_fwd_cols(const cpx<T>* T1, int H, int K, int Qh, int Qs, cpx<T>* F, const Tw<T>& tw,
                                   const DevStatus* st, int conditional, T out_scale, cudaStream_t s) {
    using C = ColCfg<T, P>;
    auto kern = k_fwd_cols<T, P>;
    cudaError_t e = ensure_smem(kern, C::smem(P));
    if (e != cudaSuccess) return e;
    dim3 grid((Qh + C::TPB - 1) / C::TPB, K);
    kern<<<grid, C::THREADS, C::smem(H), s>>>(T1, H, K, Qh, Qs, F, tw, st, conditional, out_scale);
    return cudaGetLastError();
}

template <typename T, int P>
static cudaError_t launch_pair_cols(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    using C = PairColsCfg<T, P>;
    auto kern = k_pair_cols<T, P>;
    const size_t smem = pair_cols_smem<T, P>();
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
    const long long items = (long long)g.KA * g.KB * ((g.Qh + C::TPB - 1) / C::TPB);
    const long long slots = a.num_sms > 0 ? (long long)per_sm * a.num_sms : items;
    const int grid = (int)(items < slots ? items : slots);
    e = cudaMemsetAsync(a.work_ctr, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    kern<<<grid, C::THREADS, smem, s>>>(a.FA, a.FB, g.KA, g.KB, g.Qh, g.HA, g.HB, g.R, g.Qs, g.r0, g.r1, a.Y, a.tw,
                                        a.st, a.conditional, a.work_ctr);
    return cudaGetLastError();
}

template <typename T, int Q>
static cudaError_t launch_pair_rows(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    using C = RowCfg<T, Q>;
    if constexpr (sizeof(T) == 4 && (Q == 1024 || Q == 2048)) {
        if (a.tm_cols > 0) {
            auto kern = k_pair_rows_tm<Q>;
            cudaError_t e = ensure_smem(kern, RowTmCfg<Q>::SMEM);
            if (e != cudaSuccess) return e;
            kern<<<a.rows_grid, RowTmCfg<Q>::THREADS, RowTmCfg<Q>::SMEM, s>>>(a.Y, g, a.tw, a.mi, a.n, a.counts, a.st,
                                                                             a.tm_cols);
            return cudaGetLastError();
        }
    }
    const size_t smem = pair_rows_smem<T, Q>(g.KB, a.cb_smem);
    if (a.cb_smem) {
        auto kern = k_pair_rows<T, Q, true>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<a.rows_grid, C::THREADS, smem, s>>>(a.Y, g, a.tw, a.cb_global, a.mi, a.n, a.counts, a.st,
                                                   a.prec_slot, a.conditional);
    } else {
        auto kern = k_pair_rows<T, Q, false>;
        cudaError_t e = ensure_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<a.rows_grid, C::THREADS, smem, s>>>(a.Y, g, a.tw, a.cb_global, a.mi, a.n, a.counts, a.st,
                                                   a.prec_slot, a.conditional);
    }
    return cudaGetLastError();
}

struct ProfScope {
    Profiler* p;
    cudaStream_t s;
    ProfScope(Profiler* p_, const char* name, cudaStream_t s_) : p(p_), s(s_) { if (p) p->begin(name, s); }
    ~ProfScope() { if (p) p->end(s); }
};

template <typename T>
cudaError_t run_pipeline(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    constexpr bool f32 = sizeof(T) == 4;
    constexpr bool split = std::is_same<T, df32>::value;
    const unsigned stg = a.stages ? a.stages : STAGE_ALL;
    if (stg & STAGE_FWD_A) {
        CMIF_SIZE_SWITCH(g.Q, {
            ProfScope ps(a.prof, f32 ? "fwd_rows_A_f32" : split ? "fwd_rows_A_s32" : "fwd_rows_A_f64", s);
            e = (launch_fwd_rows<T, SZ>(a.A, a.MA, g.HA, g.WA, g.KA, g.Qs, a.T1A, a.tw, a.st, a.conditional, s));
        } if (e != cudaSuccess) return e);
        CMIF_SIZE_SWITCH(g.P, {
            ProfScope ps(a.prof, f32 ? "fwd_cols_A_f32" : split ? "fwd_cols_A_s32" : "fwd_cols_A_f64", s);
            e = (launch_fwd_cols<T, SZ>(a.T1A, g.HA, g.KA, g.Qh, g.Qs, a.FA, a.tw, a.st, a.conditional, T(1), s));
        } if (e != cudaSuccess) return e);
    }
    if (stg & STAGE_FWD_B) {
        CMIF_SIZE_SWITCH(g.Q, {
            ProfScope ps(a.prof, f32 ? "fwd_rows_B_f32" : split ? "fwd_rows_B_s32" : "fwd_rows_B_f64", s);
            e = (launch_fwd_rows<T, SZ>(a.B, a.MB, g.HB, g.WB, g.KB, g.Qs, a.T1B, a.tw, a.st, a.conditional, s));
        } if (e != cudaSuccess) return e);
        CMIF_SIZE_SWITCH(g.P, {
            ProfScope ps(a.prof, f32 ? "fwd_cols_B_f32" : split ? "fwd_cols_B_s32" : "fwd_cols_B_f64", s);
            // B's spectra carry the 1/(P Q) of the unnormalised inverse transform (a power of two: exact)
            e = (launch_fwd_cols<T, SZ>(a.T1B, g.HB, g.KB, g.Qh, g.Qs, a.FB, a.tw, a.st, a.conditional,
                                        T(1.0 / ((double)g.P * (double)g.Q)), s));
        } if (e != cudaSuccess) return e);
    }
    if (stg & STAGE_PAIRS) {
        CMIF_SIZE_SWITCH(g.P, {
            ProfScope ps(a.prof, f32 ? "pair_cols_f32" : split ? "pair_cols_s32" : "pair_cols_f64", s);
            e = (launch_pair_cols<T, SZ>(g, a, s));
        } if (e != cudaSuccess) return e);
        CMIF_SIZE_SWITCH(g.Q, {
            ProfScope ps(a.prof, f32 ? "pair_rows_f32" : split ? "pair_rows_s32" : "pair_rows_f64", s);
            e = (launch_pair_rows<T, SZ>(g, a, s));
        } if (e != cudaSuccess) return e);
    }
    return cudaSuccess;
}

template <typename T>
size_t rows_smem_bytes(int Q, int KB, bool cb_smem) {
    size_t out = 0;
    auto f = [&]() -> cudaError_t {
        CMIF_SIZE_SWITCH(Q, out = pair_rows_smem<T, SZ>(KB, cb_smem));
        return cudaSuccess;
    };
    f();
    return out;
}

template <typename T>
int rows_threads(int Q) {
    int out = 0;
    auto f = [&]() -> cudaError_t {
        CMIF_SIZE_SWITCH(Q, out = RowCfg<T, SZ>::THREADS);
        return cudaSuccess;
    };
    f();
    return out;
}

template <typename T>
cudaError_t rows_max_blocks_per_sm(int Q, int KB, bool cb_smem, int* out) {
    const size_t smem = rows_smem_bytes<T>(Q, KB, cb_smem);
    CMIF_SIZE_SWITCH(Q, {
        if (cb_smem) {
            auto kern = k_pair_rows<T, SZ, true>;
            cudaError_t e = ensure_smem(kern, smem);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, RowCfg<T, SZ>::THREADS, smem);
        } else {
            auto kern = k_pair_rows<T, SZ, false>;
            cudaError_t e = ensure_smem(kern, smem);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, RowCfg<T, SZ>::THREADS, smem);
        }
    });
    return cudaSuccess;
}

#ifdef CMIF_DEFINE_TM_HELPERS
int rows_tm_cols(int Q, int KB) {
    int U = 0;
    if (Q == 2048) U = RowTmCfg<2048>::U;
    else if (Q == 1024) U = RowTmCfg<1024>::U;
    else return 0;
    const int need = tm_cols_needed(KB, U);
    return need <= 512 ? tm_alloc_cols(need) : 0;
}

cudaError_t rows_tm_max_blocks_per_sm(int Q, int* out) {
    if (Q == 2048) {
        cudaError_t e = ensure_smem(k_pair_rows_tm<2048>, RowTmCfg<2048>::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pair_rows_tm<2048>, RowTmCfg<2048>::THREADS,
                                                             RowTmCfg<2048>::SMEM);
    }
    if (Q == 1024) {
        cudaError_t e = ensure_smem(k_pair_rows_tm<1024>, RowTmCfg<1024>::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pair_rows_tm<1024>, RowTmCfg<1024>::THREADS,
                                                             RowTmCfg<1024>::SMEM);
    }
    *out = 0;
    return cudaSuccess;
}
#endif

#define CMIF_INSTANTIATE(T)                                                             \
    template cudaError_t run_pipeline<T>(const Geom&, const PipeArgs<T>&, cudaStream_t); \
    template size_t rows_smem_bytes<T>(int, int, bool);                                  \
    template int rows_threads<T>(int);                                                   \
    template cudaError_t rows_max_blocks_per_sm<T>(int, int, bool, int*);

}  // namespace cmif
