// The launch sequence of one CMIF map, dispatched on the run-time transform
// sizes to the per-size entry points (compiled in the kernels_*.cu units).
#include <type_traits>
#include "pipeline.cuh"

namespace cmif {

namespace {
struct ProfScope {
    Profiler* p;
    cudaStream_t s;
    ProfScope(Profiler* p_, const char* name, cudaStream_t s_) : p(p_), s(s_) { if (p) p->begin(name, s); }
    ~ProfScope() { if (p) p->end(s); }
};
}  // namespace

template <typename T>
cudaError_t run_pipeline(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    constexpr bool f32 = sizeof(T) == 4;
    constexpr bool split = std::is_same<T, df32>::value;
    const unsigned stg = a.stages ? a.stages : STAGE_ALL;
    // A's and B's forward transforms are independent: with a second stream, A's run
    // on it, forked from s before and joined back into s after B's
    const bool fork = (stg & STAGE_FWD_A) && (stg & STAGE_FWD_B) && a.aux && a.ev_fork && a.ev_join;
    const cudaStream_t sa = fork ? a.aux : s;
    if (fork) {
        e = cudaEventRecord(a.ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a.aux, a.ev_fork, 0);
        if (e != cudaSuccess) return e;
    }
    if (stg & STAGE_FWD_A) {
        CMIF_SIZE_SWITCH_T(T, g.Q, {
            ProfScope ps(a.prof, f32 ? "fwd_rows_A_f32" : split ? "fwd_rows_A_s32" : "fwd_rows_A_f64", sa);
            e = Sized<T, SZ>::fwd_rows(g, a, false, sa);
        } if (e != cudaSuccess) return e);
        CMIF_SIZE_SWITCH_T(T, g.P, {
            ProfScope ps(a.prof, f32 ? "fwd_cols_A_f32" : split ? "fwd_cols_A_s32" : "fwd_cols_A_f64", sa);
            e = Sized<T, SZ>::fwd_cols(g, a, false, sa);
        } if (e != cudaSuccess) return e);
    }
    if (stg & STAGE_FWD_B) {
        CMIF_SIZE_SWITCH_T(T, g.Q, {
            ProfScope ps(a.prof, f32 ? "fwd_rows_B_f32" : split ? "fwd_rows_B_s32" : "fwd_rows_B_f64", s);
            e = Sized<T, SZ>::fwd_rows(g, a, true, s);
        } if (e != cudaSuccess) return e);
        CMIF_SIZE_SWITCH_T(T, g.P, {
            ProfScope ps(a.prof, f32 ? "fwd_cols_B_f32" : split ? "fwd_cols_B_s32" : "fwd_cols_B_f64", s);
            e = Sized<T, SZ>::fwd_cols(g, a, true, s);
        } if (e != cudaSuccess) return e);
    }
    if (fork) {
        e = cudaEventRecord(a.ev_join, a.aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, a.ev_join, 0);
        if (e != cudaSuccess) return e;
    }
    if (stg & STAGE_COLS) {
        CMIF_SIZE_SWITCH_T(T, g.P, {
            ProfScope ps(a.prof, f32 ? "pair_cols_f32" : split ? "pair_cols_s32" : "pair_cols_f64", s);
            e = Sized<T, SZ>::pair_cols(g, a, s);
        } if (e != cudaSuccess) return e);
    }
    if (stg & STAGE_ROWS) {
        if (a.weighted) {
            CMIF_SIZE_SWITCH_T(T, g.Q, {
                ProfScope ps(a.prof, "pair_rows_weighted_f64", s);
                e = Sized<T, SZ>::pair_rows_w(g, a, s);
            } if (e != cudaSuccess) return e);
        } else {
            CMIF_SIZE_SWITCH_T(T, g.Q, {
                ProfScope ps(a.prof, f32 ? "pair_rows_f32" : split ? "pair_rows_s32" : "pair_rows_f64", s);
                e = Sized<T, SZ>::pair_rows(g, a, s);
            } if (e != cudaSuccess) return e);
        }
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t run_pair_counts(const Geom& g, const PipeArgs<T>& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    constexpr bool split = std::is_same<T, df32>::value;
    CMIF_SIZE_SWITCH(g.P, {
        ProfScope ps(a.prof, split ? "pair_cols_list_s32" : "pair_cols_list_f64", s);
        e = Sized<T, SZ>::pair_cols(g, a, s);
    } if (e != cudaSuccess) return e);
    CMIF_SIZE_SWITCH(g.Q, {
        ProfScope ps(a.prof, split ? "pair_counts_s32" : "pair_counts_f64", s);
        e = Sized<T, SZ>::pair_rows_counts(g, a, s);
    } if (e != cudaSuccess) return e);
    return cudaSuccess;
}
template cudaError_t run_pair_counts<double>(const Geom&, const PipeArgs<double>&, cudaStream_t);
template cudaError_t run_pair_counts<df32>(const Geom&, const PipeArgs<df32>&, cudaStream_t);

template <typename T>
size_t rows_smem_bytes(int Q, int KB, bool cb_smem) {
    size_t out = 0;
    auto f = [&]() -> cudaError_t {
        CMIF_SIZE_SWITCH_T(T, Q, out = Sized<T, SZ>::rows_smem(KB, cb_smem));
        return cudaSuccess;
    };
    f();
    return out;
}

template <typename T>
int rows_threads(int Q) {
    int out = 0;
    auto f = [&]() -> cudaError_t {
        CMIF_SIZE_SWITCH_T(T, Q, out = Sized<T, SZ>::rows_threads());
        return cudaSuccess;
    };
    f();
    return out;
}

template <typename T>
cudaError_t rows_max_blocks_per_sm(int Q, int KB, bool cb_smem, int* out) {
    CMIF_SIZE_SWITCH_T(T, Q, return Sized<T, SZ>::rows_max_blocks(KB, cb_smem, out));
    return cudaSuccess;
}

int rows_tm_cols(int Q, int KB) {
    int out = 0;
    auto f = [&]() -> cudaError_t {
        CMIF_SIZE_SWITCH_T(float, Q, out = Sized<float, SZ>::tm_cols(KB));
        return cudaSuccess;
    };
    f();
    return out;
}

cudaError_t rows_w_max_blocks_per_sm(int Q, int* out) {
    *out = 0;
    CMIF_SIZE_SWITCH(Q, return Sized<double, SZ>::rows_w_max_blocks(out));
    return cudaSuccess;
}

cudaError_t rows_tm_max_blocks_per_sm(int Q, int* out) {
    *out = 0;
    CMIF_SIZE_SWITCH_T(float, Q, return Sized<float, SZ>::tm_max_blocks(out));
    return cudaSuccess;
}

#define CMIF_INSTANTIATE(T)                                                             \
    template cudaError_t run_pipeline<T>(const Geom&, const PipeArgs<T>&, cudaStream_t); \
    template size_t rows_smem_bytes<T>(int, int, bool);                                  \
    template int rows_threads<T>(int);                                                   \
    template cudaError_t rows_max_blocks_per_sm<T>(int, int, bool, int*);
CMIF_INSTANTIATE(float)
CMIF_INSTANTIATE(double)
CMIF_INSTANTIATE(df32)
#undef CMIF_INSTANTIATE

}  // namespace cmif
