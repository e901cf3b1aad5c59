// Launch sequence of one CMIF map for one precision (FP32 or FP64 transforms).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include "kernels.cuh"
#include "profiler.h"

namespace cmif {

template <typename T>
struct PipeArgs {
    const int32_t* A;
    const uint8_t* MA;
    const int32_t* B;
    const uint8_t* MB;
    cpx<T>* T1A;  // [K_A][H_A][Qs]  row spectra of A's level sets
    cpx<T>* T1B;  // [K_B][H_B][Qs]
    cpx<T>* FA;   // [K_A][Qh][P]    2-D half spectra, column-contiguous
    cpx<T>* FB;   // [K_B][Qh][P]
    cpx<T>* Y;    // [K_A*K_B][R][Qs] column-inverted products, output rows only
    float* cb_global;  // [rows_grid][K_B][Q] when !cb_smem
    int* work_ctr;     // item counter of the pair-column kernel (zeroed before each launch)
    Tw<T> tw;
    double* mi;
    int32_t* n;
    int32_t* counts;
    DevStatus* st;
    int prec_slot;    // 0: FP32 residual slot, 1: FP64
    int conditional;  // run only when STATUS_ESCALATE is set (AUTO re-run)
    int rows_grid;    // persistent grid of the row/epilogue kernel
    int num_sms;      // SMs of the device (persistent grid of the pair-column kernel)
    int nmi;          // the map holds NMI = (H_A + H_B) / H_AB instead of MI
    // spatially weighted MI (FP64 plans): weight images replace the masks
    const double* WA;  // [H_A][W_A] or nullptr
    const double* WB;  // [H_B][W_B] or nullptr
    int weighted;      // run the weighted row kernel (real counts, no rounding)
    double* cbw;       // [rows_grid_w][K_B][Q] B-marginals of the weighted row kernel
    double* nw;        // weighted N map [R][C]
    int rows_grid_w;   // persistent grid of the weighted row kernel
    bool cb_smem;     // B-marginal accumulators in shared memory
    Profiler* prof;   // optional launch timing (nullptr = off)
    int tm_cols;      // > 0: use the TMEM / TMA row kernel with this many TMEM columns
    int col_m;        // column transforms' lanes per group: 0 = the default (32 for FP32), 16 = the
                      // 16-lane variant (FP32, P >= 1024); the spectra layout follows it, so the
                      // forward and pair column kernels of one map must use the same value
    int cols_bps;     // persistent blocks per SM of the pair-column kernel (0: as many as fit)
    int wait_polls;   // poll limit of the TMEM row kernel's bounded waits (0: the default)
    int withhold_row; // diagnostics: output row whose first bulk copy is withheld (-1: none)
    unsigned stages;  // STAGE_* bits: which parts of the sequence to launch
    // optional second stream and events: A's and B's forward transforms run side by side
    // (fork from and join back into the call's stream; graph capture records the branch)
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_join;
    // per-pair precision (CMIF_AUTO): all nullable / 0 when unused
    int* popA;                  // [K_A] label pixel counts of A, added by the forward row kernel
    int* popB;                  // [K_B]
    const unsigned char* needA; // [K_A] planes to transform (entry 1), others skipped
    const unsigned char* needB; // [K_B]
    const int* plist;           // list mode of the pair kernels: the list of pairs (a * K_B + b)
    const int* lrange;          // [2]: entries [lrange[0], lrange[1]) of plist belong to this stage
    int chunk_off, chunk_cap;   // this launch takes entries lrange[0] + chunk_off .. + chunk_cap
    int32_t* ov;                // [list slot][R][Q] exact counts of listed pairs (written by the second tier)
    const int* ov_slot;         // [K_A * K_B] list slot of a pair, -1: the FP32 counts stand
    unsigned* pair_res;         // [K_A * K_B] largest FP32 residual of each pair (float bits)
};

enum : unsigned {
    STAGE_FWD_A = 1u,   // level-set transforms of A
    STAGE_FWD_B = 2u,   // level-set transforms of B
    STAGE_COLS = 4u,    // pair product and inverse column transforms
    STAGE_ROWS = 8u,    // inverse row transforms and the epilogue
    STAGE_PAIRS = 12u,  // both pair stages
    STAGE_ALL = 15u,
};

// The transform sizes the kernels are compiled for: P, Q = 2^k (16 .. 4096) in
// every precision, and 3 * 2^k (96 .. 3072) for FP32 transforms.
template <typename T>
constexpr bool kMixedSizes = std::is_same<T, float>::value;
#define CMIF_MIXED_CASE(TT, V, ...)                                   \
    case V: {                                                          \
        constexpr int SZ = V;                                          \
        if constexpr (kMixedSizes<TT>) { __VA_ARGS__; }                \
        else { return cudaErrorInvalidValue; }                         \
    } break;
// Power-of-two sizes and, for FP32 (TT = float), the 3 * 2^k ones.
#define CMIF_SIZE_SWITCH_T(TT, N, ...)                                \
    switch (N) {                                                      \
        case 16: { constexpr int SZ = 16; __VA_ARGS__; } break;     \
        case 32: { constexpr int SZ = 32; __VA_ARGS__; } break;     \
        case 64: { constexpr int SZ = 64; __VA_ARGS__; } break;     \
        case 128: { constexpr int SZ = 128; __VA_ARGS__; } break;   \
        case 256: { constexpr int SZ = 256; __VA_ARGS__; } break;   \
        case 512: { constexpr int SZ = 512; __VA_ARGS__; } break;   \
        case 1024: { constexpr int SZ = 1024; __VA_ARGS__; } break; \
        case 2048: { constexpr int SZ = 2048; __VA_ARGS__; } break; \
        case 4096: { constexpr int SZ = 4096; __VA_ARGS__; } break; \
        CMIF_MIXED_CASE(TT, 96, __VA_ARGS__)                          \
        CMIF_MIXED_CASE(TT, 192, __VA_ARGS__)                         \
        CMIF_MIXED_CASE(TT, 384, __VA_ARGS__)                         \
        CMIF_MIXED_CASE(TT, 768, __VA_ARGS__)                         \
        CMIF_MIXED_CASE(TT, 1536, __VA_ARGS__)                        \
        CMIF_MIXED_CASE(TT, 3072, __VA_ARGS__)                        \
        default: return cudaErrorInvalidValue;                        \
    }

// The power-of-two transform sizes (P, Q = 16 .. 4096).
#define CMIF_SIZE_SWITCH(N, ...)                                     \
    switch (N) {                                                      \
        case 16: { constexpr int SZ = 16; __VA_ARGS__; } break;     \
        case 32: { constexpr int SZ = 32; __VA_ARGS__; } break;     \
        case 64: { constexpr int SZ = 64; __VA_ARGS__; } break;     \
        case 128: { constexpr int SZ = 128; __VA_ARGS__; } break;   \
        case 256: { constexpr int SZ = 256; __VA_ARGS__; } break;   \
        case 512: { constexpr int SZ = 512; __VA_ARGS__; } break;   \
        case 1024: { constexpr int SZ = 1024; __VA_ARGS__; } break; \
        case 2048: { constexpr int SZ = 2048; __VA_ARGS__; } break; \
        case 4096: { constexpr int SZ = 4096; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                        \
    }

// Entry points of one (precision, transform size).  The definitions
// (pipeline_impl.cuh) are instantiated explicitly in the kernels_<prec>_<sizes>.cu
// units, so that the kernels of different sizes compile in parallel;
// pipeline.cu dispatches on the run-time size.
template <typename T, int SZ>
struct Sized {
    static cudaError_t fwd_rows(const Geom& g, const PipeArgs<T>& a, bool b_side, cudaStream_t s);  // Q = SZ
    static cudaError_t fwd_cols(const Geom& g, const PipeArgs<T>& a, bool b_side, cudaStream_t s);  // P = SZ
    static cudaError_t pair_cols(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);              // P = SZ
    static cudaError_t pair_rows(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);              // Q = SZ
    static cudaError_t pair_rows_counts(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);       // Q = SZ, list mode
    static size_t rows_smem(int KB, bool cb_smem);
    static int rows_threads();
    static cudaError_t rows_max_blocks(int KB, bool cb_smem, int* out);
    static int tm_cols(int KB);                 // 0 unless the TMEM row kernel applies (FP32, Q = 512 / 1024 / 2048)
    static cudaError_t tm_max_blocks(int* out);
    static cudaError_t pair_rows_w(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);  // FP64 only
    static size_t rows_w_smem();
    static cudaError_t rows_w_max_blocks(int* out);
};

template <typename T>
cudaError_t run_pipeline(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);
// The Tensor-Memory row kernel over several units (FP32, Q = 512, 1024 or 2048).
template <int Q, bool NMI>
cudaError_t launch_rows_tm_units(const Geom& g, const PipeArgs<float>& a, cudaStream_t s);
// List mode of the second precision: pair products and inverse column transforms of
// the chunk's listed pairs (into a.Y), then their exact counts (into a.ov).
template <typename T>
cudaError_t run_pair_counts(const Geom& g, const PipeArgs<T>& a, cudaStream_t s);

// Per-precision facts the host needs at plan time.
template <typename T>
size_t rows_smem_bytes(int Q, int KB, bool cb_smem);
template <typename T>
int rows_threads(int Q);
template <typename T>
cudaError_t rows_max_blocks_per_sm(int Q, int KB, bool cb_smem, int* out);
// TMEM columns the TMEM / TMA row kernel needs for (Q, K_B), or 0 when it does not apply.
int rows_tm_cols(int Q, int KB);
cudaError_t rows_tm_max_blocks_per_sm(int Q, int* out);
// The weighted (SWMI) row kernel: its occupancy (FP64).
cudaError_t rows_w_max_blocks_per_sm(int Q, int* out);

}  // namespace cmif
