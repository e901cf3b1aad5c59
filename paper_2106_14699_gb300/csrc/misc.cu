// Peak search (Alg. 1), status bookkeeping and twiddle tables.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "misc.h"

namespace cmif {

// ---------------------------------------------------------------------------
// gamma-gated argmax (Alg. 1): N_cal = gamma * max_chi N; chi* maximises MI
// among shifts with N >= N_cal; ties go to the lowest map index.
__device__ __forceinline__ bool better(double m1, long long i1, double m2, long long i2) {
    return m1 > m2 || (m1 == m2 && i1 < i2);
}

// Scans the search window rows [r0, r1) x columns [c0, c1) of the (R x Cout) maps;
// indices stay row-major map indices (ties: lowest).  NT: int32_t N (counts) or
// double N (weighted maps, max N from max_nw_bits).
__device__ __forceinline__ double max_n_of(const DevStatus* st, const int32_t*) { return (double)st->max_n; }
__device__ __forceinline__ double max_n_of(const DevStatus* st, const double*) {
    return __longlong_as_double((long long)st->max_nw_bits);
}
__device__ __forceinline__ int32_t n_record(int32_t n) { return n; }
__device__ __forceinline__ int32_t n_record(double n) { return (int32_t)fmin(rint(n), 2147483647.0); }

// Units (blockIdx.y): map u starts unit_rc elements further on, its max N comes
// from maxn_u[u] and its partials from parts + u * gridDim.x.
template <typename NT>
__global__ void k_peak_partial(const double* __restrict__ mi, const NT* __restrict__ n, int Cout, int r0, int r1,
                               int c0, int c1, const DevStatus* __restrict__ st, double gamma,
                               PeakPart* __restrict__ parts, long long unit_rc, const int* __restrict__ maxn_u) {
    mi += blockIdx.y * unit_rc;
    n += blockIdx.y * unit_rc;
    parts += (size_t)blockIdx.y * gridDim.x;
    const double thr = gamma * (maxn_u ? (double)maxn_u[blockIdx.y] : max_n_of(st, n));
    double bm = -INFINITY;
    long long bi = -1;
    // rows of the window over the blocks, columns over the threads (no index division;
    // the result does not depend on the visiting order: ties go to the lowest index)
    for (int r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const long long base = (long long)r * Cout;
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const long long i = base + c;
            if ((double)n[i] >= thr) {
                const double m = mi[i];
                if (bi < 0 || better(m, i, bm, bi)) { bm = m; bi = i; }
            }
        }
    }
    __shared__ double sm_m[32];
    __shared__ long long sm_i[32];
    for (int off = 16; off > 0; off >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, bm, off);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (oi >= 0 && (bi < 0 || better(om, oi, bm, bi))) { bm = om; bi = oi; }
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) { sm_m[w] = bm; sm_i[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k)
            if (sm_i[k] >= 0 && (bi < 0 || better(sm_m[k], sm_i[k], bm, bi))) { bm = sm_m[k]; bi = sm_i[k]; }
        parts[blockIdx.x] = {bm, bi};
    }
}

// R2 > 0 (volumes): the map rows are (depth offset, row) pairs, depth-offset
// major; the record's first field then holds the depth offset dz.
// Units (blockIdx.x): unit u reads its partials and map and writes record u.
template <typename NT>
__global__ void k_peak_final(const PeakPart* __restrict__ parts, int nparts, const double* __restrict__ mi,
                             const NT* __restrict__ n, int HA, int WA, int Cout, int angle_idx, int R2, int DA,
                             void* __restrict__ peak_out, long long unit_rc) {
    parts += (size_t)blockIdx.x * nparts;
    mi += blockIdx.x * unit_rc;
    n += blockIdx.x * unit_rc;
    peak_out = reinterpret_cast<PeakRec*>(peak_out) + blockIdx.x;
    angle_idx += blockIdx.x;
    double bm = -INFINITY;
    long long bi = -1;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x)
        if (parts[k].idx >= 0 && (bi < 0 || better(parts[k].mi, parts[k].idx, bm, bi))) { bm = parts[k].mi; bi = parts[k].idx; }
    __shared__ double sm_m[32];
    __shared__ long long sm_i[32];
    for (int off = 16; off > 0; off >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, bm, off);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (oi >= 0 && (bi < 0 || better(om, oi, bm, bi))) { bm = om; bi = oi; }
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) { sm_m[w] = bm; sm_i[w] = bi; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 1; k < nw; ++k)
        if (sm_i[k] >= 0 && (bi < 0 || better(sm_m[k], sm_i[k], bm, bi))) { bm = sm_m[k]; bi = sm_i[k]; }
    PeakRec* p = reinterpret_cast<PeakRec*>(peak_out);
    if (bi < 0) { *p = {-1, 0, 0, 0, 0.0}; return; }
    const long long row = bi / Cout;
    p->angle_idx = R2 > 0 ? (int)(row / R2) - (DA - 1) : angle_idx;
    p->dy = (int)(R2 > 0 ? row % R2 : row) - (HA - 1);
    p->dx = (int)(bi % Cout) - (WA - 1);
    p->n = n_record(n[bi]);  // weighted maps: N rounded to an integer
    p->mi = bm;
}

// ---------------------------------------------------------------------------
// Nearest-neighbour rotation of the floating image for Alg. 1's rotation grid
// (Sec. 3.6: NN interpolation because the labels are categorical).  Output
// pixel (i, j) takes the source  col = c_col + u cos - v sin,
// row = c_row + u sin + v cos  (u = j - c_col, v = i - c_row, c = ((H-1)/2, (W-1)/2)),
// each rounded half away from zero; the output mask is 1 iff the source lies
// in B and M_B(source) = 1, else label and mask are 0.
__global__ void k_warp_nn(const int32_t* __restrict__ B, const uint8_t* __restrict__ MB, int H, int W, double ct,
                          double st, int32_t* __restrict__ Bo, uint8_t* __restrict__ Mo) {
    const long long n = (long long)H * W;
    const double cr = 0.5 * (H - 1), cc = 0.5 * (W - 1);
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o / W), j = (int)(o - (long long)i * W);
        const double u = j - cc, v = i - cr;
        const double xs = cc + u * ct - v * st;
        const double ys = cr + u * st + v * ct;
        const long long si = (long long)round(ys), sj = (long long)round(xs);
        int32_t lab = 0;
        uint8_t m = 0;
        if (si >= 0 && si < H && sj >= 0 && sj < W) {
            const long long src = si * W + sj;
            if (!MB || MB[src]) { lab = B[src]; m = 1; }
        }
        Bo[o] = lab;
        Mo[o] = m;
    }
}

// Several angles at once (blockIdx.y = angle): outputs Bo + y * H * W, Mo + y * H * W.
__global__ void k_warp_nn_multi(const int32_t* __restrict__ B, const uint8_t* __restrict__ MB, int H, int W,
                                AngleSet as, int32_t* __restrict__ Bo, uint8_t* __restrict__ Mo) {
    const long long n = (long long)H * W;
    const double ct = as.c[blockIdx.y], st = as.s[blockIdx.y];
    Bo += blockIdx.y * n;
    Mo += blockIdx.y * n;
    const double cr = 0.5 * (H - 1), cc = 0.5 * (W - 1);
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o / W), j = (int)(o - (long long)i * W);
        const double u = j - cc, v = i - cr;
        const double xs = cc + u * ct - v * st;
        const double ys = cr + u * st + v * ct;
        const long long si = (long long)round(ys), sj = (long long)round(xs);
        int32_t lab = 0;
        uint8_t m = 0;
        if (si >= 0 && si < H && sj >= 0 && sj < W) {
            const long long src = si * W + sj;
            if (!MB || MB[src]) { lab = B[src]; m = 1; }
        }
        Bo[o] = lab;
        Mo[o] = m;
    }
}

cudaError_t launch_warp_nn_multi(const int32_t* B, const uint8_t* MB, int H, int W, const double* theta, int n_angles,
                                 int32_t* Bo, uint8_t* Mo, cudaStream_t s) {
    if (n_angles < 1 || n_angles > kMaxUnits) return cudaErrorInvalidValue;
    AngleSet as{};
    for (int i = 0; i < n_angles; ++i) { as.c[i] = std::cos(theta[i]); as.s[i] = std::sin(theta[i]); }
    const long long n = (long long)H * W;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    k_warp_nn_multi<<<dim3(blocks, n_angles), 256, 0, s>>>(B, MB, H, W, as, Bo, Mo);
    return cudaGetLastError();
}

cudaError_t launch_warp_nn(const int32_t* B, const uint8_t* MB, int H, int W, double theta, int32_t* Bo, uint8_t* Mo,
                           cudaStream_t s) {
    const long long n = (long long)H * W;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_warp_nn<<<blocks, 256, 0, s>>>(B, MB, H, W, std::cos(theta), std::sin(theta), Bo, Mo);
    return cudaGetLastError();
}

// Fold one map's device status into the call's running total.
__global__ void k_merge_status(const DevStatus* __restrict__ m, DevStatus* __restrict__ tot, int slot_default) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (slot_default == 2) {  // per-pair precision: FP32 pairs and second-precision pairs kept apart
            tot->res_bits[0] = max(tot->res_bits[0], m->res_bits[0]);
            tot->res_bits[1] = max(tot->res_bits[1], m->res_bits[1]);
        } else {
            tot->res_bits[0] = max(tot->res_bits[0], m->res_bits[slot_default]);  // the authoritative pass
        }
        tot->flags |= m->flags;
        tot->escalations += m->escalations;
        tot->predicted += m->predicted;
        tot->max_n = max(tot->max_n, m->max_n);
    }
}

cudaError_t launch_merge_status(const DevStatus* m, DevStatus* tot, int slot_default, cudaStream_t s) {
    k_merge_status<<<1, 32, 0, s>>>(m, tot, slot_default);
    return cudaGetLastError();
}

// Alg. 1 over transforms: the per-transform bests sorted by MI (descending),
// earlier transform first among equals; out[0] is Alg. 1's choice when its MI
// is > 0 (I starts at 0, strict >).  Slots beyond n get angle_idx = -1.
__global__ void k_topk(const PeakRec* __restrict__ peaks, int n, int k, PeakRec* __restrict__ out) {
    __shared__ unsigned char used[4096];
    for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
    __syncwarp();
    for (int q = 0; q < k; ++q) {
        double bm = -INFINITY;
        int bi = -1;
        for (int i = threadIdx.x; i < n; i += 32) {
            if (used[i] || peaks[i].angle_idx < 0) continue;
            const double m = peaks[i].mi;
            if (bi < 0 || m > bm || (m == bm && i < bi)) { bm = m; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double om = __shfl_xor_sync(0xffffffffu, bm, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (oi >= 0 && (bi < 0 || om > bm || (om == bm && oi < bi))) { bm = om; bi = oi; }
        }
        if (threadIdx.x == 0) {
            if (bi >= 0) { out[q] = peaks[bi]; used[bi] = 1; }
            else out[q] = {-1, 0, 0, 0, 0.0};
        }
        __syncwarp();
    }
}

cudaError_t launch_topk(const void* peaks, int n, int k, void* out, cudaStream_t s) {
    k_topk<<<1, 32, 0, s>>>(reinterpret_cast<const PeakRec*>(peaks), n, k, reinterpret_cast<PeakRec*>(out));
    return cudaGetLastError();
}

// A status word as a cmif_status code (0 OK, 2 LABEL_RANGE, 6 TIMEOUT, 5 PRECISION, in that order).
__global__ void k_status_code_of(const DevStatus* st, int32_t* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const unsigned f = st->flags;
        *out = (f & STATUS_LABEL_RANGE) ? 2 : (f & STATUS_TIMEOUT) ? 6 : (f & STATUS_PRECISION) ? 5 : 0;
    }
}

cudaError_t launch_status_code(const DevStatus* st, int32_t* out, cudaStream_t s) {
    k_status_code_of<<<1, 32, 0, s>>>(st, out);
    return cudaGetLastError();
}

// Final decision on the authoritative precision's residual (slot 2: per-pair
// precision, where both the FP32 pairs' and the second-precision pairs' count).
__global__ void k_finalize(DevStatus* st, int slot_if_escalated, int slot_default) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int slot = (st->flags & STATUS_ESCALATE) ? slot_if_escalated : slot_default;
        const unsigned r = slot == 2 ? max(st->res_bits[0], st->res_bits[1]) : st->res_bits[slot];
        if (__uint_as_float(r) >= kResidualGuard) st->flags |= STATUS_PRECISION;
    }
}

// Max N over each unit's window (units > 1: the gamma gate of Alg. 1 is per map).
__global__ void k_unit_max_n(const int32_t* __restrict__ n, int Cout, int r0, int r1, int c0, int c1,
                             long long unit_rc, int* __restrict__ maxn_u) {
    n += blockIdx.y * unit_rc;
    int m = 0;
    for (int r = r0 + blockIdx.x; r < r1; r += gridDim.x)
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) m = max(m, n[(long long)r * Cout + c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&maxn_u[blockIdx.y], m);
}

template <typename NT>
static cudaError_t launch_peak_t(const double* mi, const NT* n, const Geom& g, const DevStatus* st, double gamma,
                                 PeakPart* parts, int nparts, int angle_idx, void* peak_out, int units,
                                 const int* maxn_u, cudaStream_t s) {
    const int HA = g.HA, WA = g.WA, Cout = g.C;
    const long long unit_rc = units > 1 ? (long long)g.R2 * Cout : 0;
    k_peak_partial<NT><<<dim3(nparts, units), 256, 0, s>>>(mi, n, Cout, g.r0, g.r1, g.c0, g.c1, st, gamma, parts,
                                                           unit_rc, units > 1 ? maxn_u : nullptr);
    k_peak_final<NT><<<units, 256, 0, s>>>(parts, nparts, mi, n, HA, WA, Cout, angle_idx, g.Dz > 1 ? g.R2 : 0, g.DA,
                                             peak_out, unit_rc);
    return cudaGetLastError();
}

cudaError_t launch_peak(const double* mi, const int32_t* n, const Geom& g, const DevStatus* st, double gamma,
                        PeakPart* parts, int nparts, int angle_idx, void* peak_out, cudaStream_t s) {
    return launch_peak_t(mi, n, g, st, gamma, parts, nparts, angle_idx, peak_out, 1, nullptr, s);
}

cudaError_t launch_peak_units(const double* mi, const int32_t* n, const Geom& g, const DevStatus* st, double gamma,
                              PeakPart* parts, int nparts, int angle0, void* peaks_out, int* maxn_u,
                              cudaStream_t s) {
    // per-unit max N first (zeroed here), then the gated argmax of every unit
    cudaError_t e = cudaMemsetAsync(maxn_u, 0, (size_t)g.units * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const long long unit_rc = (long long)g.R2 * g.C;
    k_unit_max_n<<<dim3(std::max(1, nparts / 2), g.units), 256, 0, s>>>(n, g.C, g.r0, g.r1, g.c0, g.c1, unit_rc,
                                                                         maxn_u);
    return launch_peak_t(mi, n, g, st, gamma, parts, nparts, angle0, peaks_out, g.units, maxn_u, s);
}

cudaError_t launch_peak_w(const double* mi, const double* nw, const Geom& g, const DevStatus* st, double gamma,
                          PeakPart* parts, int nparts, void* peak_out, cudaStream_t s) {
    return launch_peak_t(mi, nw, g, st, gamma, parts, nparts, 0, peak_out, 1, nullptr, s);
}

cudaError_t launch_finalize(DevStatus* st, int slot_if_escalated, int slot_default, cudaStream_t s) {
    k_finalize<<<1, 32, 0, s>>>(st, slot_if_escalated, slot_default);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-pair precision of CMIF_AUTO.  The rounding of Sec. 3.2 gives exact counts
// only while every pre-rounding error stays under 0.5; the error of an FFT
// correlation of two 0/1 planes grows like u log2(PQ) sqrt(|X_a| |Y_b|) (u the
// unit roundoff, |X| the plane's pixel count), so pairs of large label areas
// need the second precision first.

// Ordered compaction of the flagged pairs of one block (1024 threads, <= 4096
// pairs): slots first + 0, 1, ... in pair order, those below cap written to the
// list (a pair beyond the cap keeps its FP32 counts); returns the number flagged.
template <typename Flag>
__device__ __forceinline__ int block_compact(Flag flag, int npairs, int first, int cap, int* __restrict__ plist,
                                             int* __restrict__ ov_slot) {
    __shared__ int s_cnt[1024];
    constexpr int PER = 4;  // 1024 threads x 4 >= 4096 pairs
    const int t = threadIdx.x;
    bool f[PER];
    int c = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = t * PER + i;
        f[i] = p < npairs && flag(p);
        c += f[i];
    }
    s_cnt[t] = c;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan
        const int v = t >= off ? s_cnt[t - off] : 0;
        __syncthreads();
        s_cnt[t] += v;
        __syncthreads();
    }
    int slot = first + s_cnt[t] - c;
    const int total = s_cnt[1023];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int p = t * PER + i;
        if (f[i]) {
            if (slot < cap) {
                plist[slot] = p;
                ov_slot[p] = slot;
            }
            ++slot;
        }
    }
    __syncthreads();
    return total;
}

// The predicate: a pair goes to the second precision up front when
// scale * sqrt(|X_a| |Y_b|) >= thr (scale = kappa u log2(PQ), thr below the guard).
// Also resets the list, the slots, the per-pair residuals and the plane masks.
__global__ void __launch_bounds__(1024) k_select_pairs(const int* __restrict__ popA, const int* __restrict__ popB,
                                                      int KA, int KB, double scale, double thr, int cap,
                                                      int* __restrict__ plist, int* __restrict__ hdr,
                                                      int* __restrict__ ov_slot, unsigned* __restrict__ pair_res,
                                                      unsigned char* __restrict__ needA,
                                                      unsigned char* __restrict__ needB, DevStatus* __restrict__ st) {
    const int npairs = KA * KB;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) { ov_slot[p] = -1; pair_res[p] = 0u; }
    for (int k = threadIdx.x; k < KA; k += blockDim.x) needA[k] = 0;
    for (int k = threadIdx.x; k < KB; k += blockDim.x) needB[k] = 0;
    __syncthreads();
    auto flag = [&](int p) {
        const double pa = popA[p / KB], pb = popB[p % KB];
        return scale * sqrt(pa * pb) >= thr;
    };
    const int n = min(block_compact(flag, npairs, 0, cap, plist, ov_slot), cap);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        needA[plist[i] / KB] = 1;
        needB[plist[i] % KB] = 1;
    }
    if (threadIdx.x == 0) {
        hdr[0] = 0;
        hdr[1] = n;
        hdr[2] = n;
        st->predicted += n;
    }
}

// The guard after the FP32 pass: pairs not yet in the list whose residual reached
// 0.25 are appended (stage 2); the planes they need that stage 1 did not transform
// are marked; the re-run of the FP32 row pass is requested, with its residual and
// max N started afresh.
__global__ void __launch_bounds__(1024) k_check_pairs(const unsigned* __restrict__ pair_res, int KA, int KB, int cap,
                                                     int* __restrict__ plist, int* __restrict__ hdr,
                                                     int* __restrict__ ov_slot, unsigned char* __restrict__ needA,
                                                     unsigned char* __restrict__ needB, DevStatus* __restrict__ st) {
    const int npairs = KA * KB;
    for (int k = threadIdx.x; k < KA; k += blockDim.x) if (needA[k] == 1) needA[k] = 2;  // done in stage 1
    for (int k = threadIdx.x; k < KB; k += blockDim.x) if (needB[k] == 1) needB[k] = 2;
    const int first = hdr[1];
    __syncthreads();
    auto flag = [&](int p) { return ov_slot[p] < 0 && __uint_as_float(pair_res[p]) >= kResidualGuard; };
    const int n = min(block_compact(flag, npairs, first, cap, plist, ov_slot), cap - first);
    for (int i = first + threadIdx.x; i < first + n; i += blockDim.x) {
        const int a = plist[i] / KB, b = plist[i] % KB;
        if (needA[a] == 0) needA[a] = 1;
        if (needB[b] == 0) needB[b] = 1;
    }
    if (threadIdx.x == 0) {
        hdr[2] = first + n;
        if (n > 0) {
            st->flags |= STATUS_ESCALATE;
            st->escalations += n;
            st->res_bits[0] = 0u;
            st->max_n = 0;
        }
    }
}

cudaError_t launch_select_pairs(const int* popA, const int* popB, int KA, int KB, double scale, double thr, int cap,
                                int* plist, int* hdr, int* ov_slot, unsigned* pair_res, unsigned char* needA,
                                unsigned char* needB, DevStatus* st, cudaStream_t s) {
    if (KA * KB > 4096 || cap < 1) return cudaErrorInvalidValue;
    k_select_pairs<<<1, 1024, 0, s>>>(popA, popB, KA, KB, scale, thr, cap, plist, hdr, ov_slot, pair_res, needA,
                                      needB, st);
    return cudaGetLastError();
}

cudaError_t launch_check_pairs(const unsigned* pair_res, int KA, int KB, int cap, int* plist, int* hdr,
                               int* ov_slot, unsigned char* needA, unsigned char* needB, DevStatus* st,
                               cudaStream_t s) {
    if (KA * KB > 4096 || cap < 1) return cudaErrorInvalidValue;
    k_check_pairs<<<1, 1024, 0, s>>>(pair_res, KA, KB, cap, plist, hdr, ov_slot, needA, needB, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Synthetic labels for timing runs (the autotuner): X[i] = hash(i, seed) mod K.
// The transforms' cost does not depend on the labels.
__global__ void k_fill_labels(int32_t* __restrict__ X, long long n, int K, unsigned seed) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)i * 2654435761u ^ seed;
        h ^= h >> 16;
        h *= 0x7feb352du;
        h ^= h >> 15;
        X[i] = (int32_t)(h % (unsigned)K);
    }
}

cudaError_t launch_fill_labels(int32_t* X, long long n, int K, unsigned seed, cudaStream_t s) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    k_fill_labels<<<blocks, 256, 0, s>>>(X, n, K, seed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The epilogue's per-count entropy term T(c) = c log2 c (Eq. finalentropy), as
// the row kernels evaluate it, for the counts c0 .. c0 + n - 1.
__global__ void k_entropy_terms(int c0, int n, long long* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = clog2c_fixed((float)(c0 + i));
}

cudaError_t launch_entropy_terms(int c0, int n, long long* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = std::min((n + 255) / 256, 4096);
    k_entropy_terms<<<blocks, 256, 0, s>>>(c0, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Twiddle tables: e^{-2 pi i k / N} evaluated in FP64 with octant symmetry
// (so mirrored entries are exact negatives / swaps), then rounded to the
// table precision.
static void host_twiddle(long long k, long long N, double* c, double* s) {
    k %= N;
    if (N <= 2) {
        *c = (k == 0) ? 1.0 : -1.0;
        *s = 0.0;
        return;
    }
    if (N % 4 != 0) {  // N = 3, 6
        const double t = 2.0 * M_PI * (double)k / (double)N;
        *c = std::cos(t);
        *s = -std::sin(t);
        return;
    }
    const long long q4 = N / 4;  // N = 2^l or 3 2^l, divisible by 4
    const long long qd = k / q4, r = k - qd * q4;
    double cu, su;
    if (2 * r <= q4) {
        const double t = 2.0 * M_PI * (double)r / (double)N;
        cu = std::cos(t);
        su = std::sin(t);
    } else {
        const double t = 2.0 * M_PI * (double)(q4 - r) / (double)N;
        cu = std::sin(t);
        su = std::cos(t);
    }
    double cc, ss;  // cos, sin of 2 pi k / N
    switch (qd) {
        case 0: cc = cu; ss = su; break;
        case 1: cc = -su; ss = cu; break;
        case 2: cc = -cu; ss = -su; break;
        default: cc = su; ss = -cu; break;
    }
    *c = cc;
    *s = -ss;  // e^{-i t}
}

void twiddle_table_f32(std::vector<float>& out, size_t off_n[14], size_t off_sq[6], size_t off_n3[12]) {
    out.clear();
    size_t n = 0;
    for (int l = 0; l < 14; ++l) {
        off_n[l] = n;
        const long long N = 1LL << l;
        for (long long k = 0; k < N; ++k, ++n) {
            double c, s;
            host_twiddle(k, N, &c, &s);
            out.push_back((float)c);
            out.push_back((float)s);
        }
    }
    for (int l = 0; l < 6; ++l) {
        off_sq[l] = n;
        const long long M = 1LL << l;
        for (long long k1 = 0; k1 < M; ++k1)
            for (long long j = 0; j < M; ++j, ++n) {
                double c, s;
                host_twiddle(j * k1, M * M, &c, &s);
                out.push_back((float)c);
                out.push_back((float)s);
            }
    }
    for (int l = 0; l < 12; ++l) {
        off_n3[l] = n;
        const long long N = 3LL << l;
        for (long long k = 0; k < N; ++k, ++n) {
            double c, s;
            host_twiddle(k, N, &c, &s);
            out.push_back((float)c);
            out.push_back((float)s);
        }
    }
}

struct DevTables {
    void* buf = nullptr;
    Tw<float> tf{};
    Tw<double> td{};
    Tw<df32> ts{};
};

static std::mutex g_tw_mu;
static DevTables g_tw[64];

cudaError_t get_twiddles(int device, Tw<float>* tf, Tw<double>* td, Tw<df32>* ts) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tw_mu);
    DevTables& t = g_tw[device];
    if (!t.buf) {
        // layout: for l = 0..13 the N = 2^l tables, then for l = 0..5 the (2^l)^2 square tables;
        // first all FP64, then all FP32.
        std::vector<double> re, im;
        std::vector<size_t> off_n(14), off_sq(6), off_n3(12);
        for (int l = 0; l < 14; ++l) {
            off_n[l] = re.size();
            const long long N = 1LL << l;
            for (long long k = 0; k < N; ++k) {
                double c, s;
                host_twiddle(k, N, &c, &s);
                re.push_back(c);
                im.push_back(s);
            }
        }
        for (int l = 0; l < 6; ++l) {
            off_sq[l] = re.size();
            const long long M = 1LL << l;
            for (long long k1 = 0; k1 < M; ++k1)
                for (long long j = 0; j < M; ++j) {
                    double c, s;
                    host_twiddle(j * k1, M * M, &c, &s);
                    re.push_back(c);
                    im.push_back(s);
                }
        }
        for (int l = 0; l < 12; ++l) {
            off_n3[l] = re.size();
            const long long N = 3LL << l;
            for (long long k = 0; k < N; ++k) {
                double c, s;
                host_twiddle(k, N, &c, &s);
                re.push_back(c);
                im.push_back(s);
            }
        }
        const size_t n = re.size();
        std::vector<double> hd(2 * n);
        std::vector<float> hf(2 * n), hs(4 * n);
        for (size_t i = 0; i < n; ++i) {
            hd[2 * i] = re[i];
            hd[2 * i + 1] = im[i];
            hf[2 * i] = (float)re[i];
            hf[2 * i + 1] = (float)im[i];
            const float rh = (float)re[i], ih = (float)im[i];
            hs[4 * i] = rh;
            hs[4 * i + 1] = (float)(re[i] - (double)rh);
            hs[4 * i + 2] = ih;
            hs[4 * i + 3] = (float)(im[i] - (double)ih);
        }
        const size_t bytes_d = 2 * n * sizeof(double), bytes_f = 2 * n * sizeof(float), bytes_s = 4 * n * sizeof(float);
        int prev = -1;
        cudaGetDevice(&prev);
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return e;
        void* buf = nullptr;
        e = cudaMalloc(&buf, bytes_d + bytes_f + bytes_s);
        if (e == cudaSuccess) e = cudaMemcpy(buf, hd.data(), bytes_d, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((char*)buf + bytes_d, hf.data(), bytes_f, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((char*)buf + bytes_d + bytes_f, hs.data(), bytes_s, cudaMemcpyHostToDevice);
        if (prev >= 0) cudaSetDevice(prev);
        if (e != cudaSuccess) {
            if (buf) cudaFree(buf);
            return e;
        }
        t.buf = buf;
        const cpx<double>* bd = reinterpret_cast<const cpx<double>*>(buf);
        const cpx<float>* bf = reinterpret_cast<const cpx<float>*>((char*)buf + bytes_d);
        const cpx<df32>* bs = reinterpret_cast<const cpx<df32>*>((char*)buf + bytes_d + bytes_f);
        for (int l = 0; l < 14; ++l) { t.td.n[l] = bd + off_n[l]; t.tf.n[l] = bf + off_n[l]; t.ts.n[l] = bs + off_n[l]; }
        for (int l = 0; l < 6; ++l) { t.td.sq[l] = bd + off_sq[l]; t.tf.sq[l] = bf + off_sq[l]; t.ts.sq[l] = bs + off_sq[l]; }
        for (int l = 0; l < 12; ++l) { t.td.n3[l] = bd + off_n3[l]; t.tf.n3[l] = bf + off_n3[l]; t.ts.n3[l] = bs + off_n3[l]; }
    }
    if (tf) *tf = t.tf;
    if (td) *td = t.td;
    if (ts) *ts = t.ts;
    return cudaSuccess;
}

}  // namespace cmif
