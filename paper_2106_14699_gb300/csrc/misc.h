// Host-side launchers of the small kernels in misc.cu.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "common.h"
#include "fft.cuh"

namespace cmif {

struct PeakPart;

// Device image of cmif_peak (include/cmif.h): same 24-byte layout.
struct PeakRec {
    int32_t angle_idx, dy, dx, n;
    double mi;
};

// Alg. 1's gamma-gated argmax over the call's search window (g.r0..g.r1, g.c0..g.c1).
cudaError_t launch_peak(const double* mi, const int32_t* n, const Geom& g, const DevStatus* st, double gamma,
                        PeakPart* parts, int nparts, int angle_idx, void* peak_out, cudaStream_t s);
// Alg. 1's gated argmax of each of g.units maps (unit u: rows u * R2 .., window per unit,
// its own max N in maxn_u[u], records peaks_out[u] with angle index angle0 + u); the
// partials need nparts * g.units records.
cudaError_t launch_peak_units(const double* mi, const int32_t* n, const Geom& g, const DevStatus* st, double gamma,
                              PeakPart* parts, int nparts, int angle0, void* peaks_out, int* maxn_u,
                              cudaStream_t s);
// The same on a weighted map (real N, max N from the status word's max_nw_bits).
cudaError_t launch_peak_w(const double* mi, const double* nw, const Geom& g, const DevStatus* st, double gamma,
                          PeakPart* parts, int nparts, void* peak_out, cudaStream_t s);
// CMIF_AUTO per-pair precision: the predicate (list stage 1) and the guard check (stage 2).
cudaError_t launch_select_pairs(const int* popA, const int* popB, int KA, int KB, double scale, double thr, int cap,
                                int* plist, int* hdr, int* ov_slot, unsigned* pair_res, unsigned char* needA,
                                unsigned char* needB, DevStatus* st, cudaStream_t s);
cudaError_t launch_check_pairs(const unsigned* pair_res, int KA, int KB, int cap, int* plist, int* hdr,
                               int* ov_slot, unsigned char* needA, unsigned char* needB, DevStatus* st,
                               cudaStream_t s);
cudaError_t launch_finalize(DevStatus* st, int slot_if_escalated, int slot_default, cudaStream_t s);
cudaError_t launch_warp_nn(const int32_t* B, const uint8_t* MB, int H, int W, double theta, int32_t* Bo, uint8_t* Mo,
                           cudaStream_t s);
// The most units (rotation angles) one launch of the stage kernels takes.
constexpr int kMaxUnits = 64;
struct AngleSet {  // passed by value to the batched warp kernel
    double c[kMaxUnits], s[kMaxUnits];
};
// NN warp of B, M_B by n_angles angles in one launch: outputs angle-major.
cudaError_t launch_warp_nn_multi(const int32_t* B, const uint8_t* MB, int H, int W, const double* theta, int n_angles,
                                 int32_t* Bo, uint8_t* Mo, cudaStream_t s);
cudaError_t launch_merge_status(const DevStatus* m, DevStatus* tot, int slot_default, cudaStream_t s);
cudaError_t launch_status_code(const DevStatus* st, int32_t* out, cudaStream_t s);
cudaError_t launch_topk(const void* peaks, int n, int k, void* out, cudaStream_t s);
// T(c) = c log2 c of the row epilogue (fixed point, units of 2^-kFixBits) for c0 .. c0 + n - 1.
cudaError_t launch_entropy_terms(int c0, int n, long long* out, cudaStream_t s);
// Synthetic labels in [0, K) for timing runs.
cudaError_t launch_fill_labels(int32_t* X, long long n, int K, unsigned seed, cudaStream_t s);
cudaError_t get_twiddles(int device, Tw<float>* tf, Tw<double>* td, Tw<df32>* ts);
// Host copy of the FP32 twiddle tables (interleaved re, im) and the entry offsets
// of each table (lengths 2^l, the (2^l)^2 squares, lengths 3 2^l).
void twiddle_table_f32(std::vector<float>& out, size_t off_n[14], size_t off_sq[6], size_t off_n3[12]);

}  // namespace cmif
