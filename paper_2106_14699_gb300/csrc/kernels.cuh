// CMIF kernels: the frequency-domain method of Sec. 3.2.
//
//   fwd_rows   : level sets L_a[X] of one label image (Sec. 3.1), two planes
//                packed per complex row FFT of length Q, unpacked into the
//                half spectra of both planes.  Also checks labels in range.
//   fwd_cols   : column FFT of length P -> 2-D half spectra F[plane][kx][ky].
//   pair_cols  : for every label pair (a, b): conj(F[L_a A]) * F[L_b B] (the
//                correlation theorem for Eq. cc), inverse column FFT -> Y.
//   pair_rows  : inverse row FFT (complex-to-real, length Q) of every pair's
//                Y row, rounded to integer joint counts C_AB^{a,b}(chi)
//                (Eq. correlationjointhisto; rounding per Sec. 3.2), fused
//                with the per-shift entropy reduction: the marginals
//                C_A^a = sum_b C_AB^{a,b}, C_B^b = sum_a C_AB^{a,b} and
//                N = sum_a C_A^a (Eq. number), and
//                MI = log2 N + (sum c log2 c (joint) - sum (marginals)) / N,
//                which is Eq. finalentropy + Eq. mientropy rearranged.  The
//                K_A*K_B count maps never reach global memory.
//   peak       : the gamma-gated argmax of Alg. 1 for one map.
#pragma once
#include <type_traits>
#include <cstdint>
#include "common.h"
#include "fft.cuh"

namespace cmif {

// ---------------------------------------------------------------------------
// c * log2(c) for an exact non-negative integer c < 2^23 held in a float, in
// fixed point (units of 2^-kFixBits) so that per-shift sums are exact, order
// independent and cheap (integer adds): c * L(c), where for c = m * 2^e,
// m in [1, 2), L(c) = e * 2^F + round(log2(m) * 2^F).  log2(m) comes from the
// MUFU lg2 approximation; the rounding to the 2^-F grid adds at most 2^-(F+1).
// The largest |L(c) 2^-F - log2 c| over every count the epilogue can meet is
// measured exhaustively through cmif_entropy_terms (include/cmif.h).
__device__ __forceinline__ long long clog2c_fixed(float c) {
    const int ci = __float_as_int(c + 8388608.0f) - 0x4B000000;
    const int bits = __float_as_int(c);
    const float lm = __log2f(__int_as_float((bits & 0x7FFFFF) | 0x3F800000));
    // 2^23 + log2(m) 2^23 lies in [2^23, 2^24], where floats are spaced 1 apart and
    // their bit patterns grow by 1 per unit: the FMA rounds log2(m) 2^23 to the
    // nearest integer and the bits give it back (no float-to-integer conversion).
    // bits & 0x7F800000 = (e + 127) 2^23.  c = 0: ci = 0, so the term is 0 (Sec. 3.2:
    // 0 log 0 = 0) whatever L is.  c = 1: m = 1 and e = 0, so L = 0.  T stays one
    // fixed function of c, so equal counts still cancel exactly between joint and
    // marginal sums.
    const int t = __float_as_int(fmaf(lm, 8388608.0f, 8388608.0f));
    const int L = ((bits & 0x7F800000) - 0x3F800000) + (t - 0x4B000000);  // e 2^23 + round(log2(m) 2^23)
    return (long long)ci * (long long)L;
}

// Nearest integer of |v| < 2^22 with two FP32 adds (the 1.5 * 2^23 shift
// leaves no fraction bits).
__device__ __forceinline__ float round_fp32(float v) { return (v + 12582912.0f) - 12582912.0f; }

// MI(chi) = (S + N log2 N) / N, where S = sum_joint c log2 c - sum_A - sum_B and
// every c log2 c term (N log2 N included) comes from clog2c_fixed, so that MI is
// exactly 0 whenever the entropies cancel exactly (e.g. a single label).
__device__ __forceinline__ double mi_finish(long long S, int N) {
    if (N <= 0) return 0.0;  // 0/0 = 0: no overlap, no information (Sec. 3.2)
    const long long Sp = S + clog2c_fixed((float)N);
    const float sh = (float)Sp;
    const long long rem = Sp - (long long)sh;
    const float sl = (float)rem;
    const float fN = (float)N;
    const float inv = 1.0f / fN;
    const float q1 = sh * inv;
    const float r1 = fmaf(-q1, fN, sh) + sl;
    const float q2 = r1 * inv;
    return ((double)q1 + (double)q2) * (1.0 / (double)(1 << kFixBits));
}

// NMI(chi) = (H_A + H_B) / H_AB (the normalised MI the paper cites next to
// MI, Sec. 2.1), from the same fixed-point sums kept apart: SJ = sum_joint c log2 c,
// SM = sum_A + sum_B.  With T(N) = N log2 N: H_A + H_B = (2 T(N) - SM) / N and
// H_AB = (T(N) - SJ) / N.  0 when N = 0 or H_AB = 0 (0/0 = 0, Sec. 3.2).
__device__ __forceinline__ double nmi_finish(long long SJ, long long SM, int N) {
    if (N <= 0) return 0.0;
    const long long TN = clog2c_fixed((float)N);
    const long long den = TN - SJ;
    if (den == 0) return 0.0;
    return (double)(2 * TN - SM) / (double)den;
}

// Per-position entropy sums of the row epilogue: MI keeps one signed sum
// (joint terms in, marginal terms out); NMI keeps the two apart.
template <bool NMI>
struct EntAcc;
template <>
struct EntAcc<false> {
    long long s;
    __device__ __forceinline__ void zero() { s = 0; }
    __device__ __forceinline__ void joint(long long t) { s += t; }
    __device__ __forceinline__ void marg(long long t) { s -= t; }
    __device__ __forceinline__ double finish(int N) const { return mi_finish(s, N); }
};
template <>
struct EntAcc<true> {
    long long j, m;
    __device__ __forceinline__ void zero() { j = 0; m = 0; }
    __device__ __forceinline__ void joint(long long t) { j += t; }
    __device__ __forceinline__ void marg(long long t) { m += t; }
    __device__ __forceinline__ double finish(int N) const { return nmi_finish(j, m, N); }
};

__device__ __forceinline__ void atomic_max_float_pos(unsigned* addr, float v) {
    atomicMax(addr, __float_as_uint(v));  // v >= 0: float order = unsigned order
}

template <typename T>
__device__ __forceinline__ T rint_t(T v);
template <>
__device__ __forceinline__ float rint_t<float>(float v) { return rintf(v); }
template <>
__device__ __forceinline__ double rint_t<double>(double v) { return rint(v); }
// nearest integer to hi + lo (|hi + lo| < 2^23): round hi, then let lo move it by one
template <>
__device__ __forceinline__ df32 rint_t<df32>(df32 v) {
    float r = rintf(v.hi);
    const float d = (v.hi - r) + v.lo;  // v.hi - r is exact
    if (d > 0.5f) r += 1.f;
    else if (d < -0.5f) r -= 1.f;
    return {r, 0.f};
}

// Map a circular shift index (0..n-1) to the output map index, or -1 when the
// shift lies in the zero-padding gap (cannot happen for in-range shifts).
__device__ __forceinline__ int circ_to_out(int s, int n, int lo_count /*H_A or W_A*/, int hi_max /*H_B-1*/) {
    if (s <= hi_max) return s + lo_count - 1;
    if (s >= n - (lo_count - 1)) return s - n + lo_count - 1;
    return -1;
}

// ---------------------------------------------------------------------------
// Team geometry for a transform of length N in precision T.
__host__ __device__ constexpr int pow2_floor(int n) { return n < 2 ? 1 : 2 * pow2_floor(n / 2); }

// MMAX caps the lanes per group (and the values per lane): the default is the
// register budget of T; a smaller one trades a radix-R step for more warps.
template <typename T, int N, int MMAX = max_m<T>()>
struct TeamGeom {
    static constexpr int M = team_m(N, MMAX);
    static constexpr int R = N / (M * M);
    static constexpr int TEAM = R * M;                                        // lanes
    static constexpr int SCRATCH = team_scratch_bytes<T, M, R>();            // bytes of FFT scratch
};

// ---------------------------------------------------------------------------
// Forward row transforms.  Block = (row y, TPB plane pairs); team t takes the
// plane pair pp = blockIdx.y * TPB + t (planes 2pp, 2pp+1).  The block first
// stages the row as one byte per pixel (the label, or kMaskedOut where the
// mask is 0; the label range is checked here), then every team builds its two
// level sets from shared memory.  With a weight image WX (spatially weighted
// MI, Sec. 3.3) the level sets carry the weight W(x) instead of 1 (weight 0 plays
// the mask's 0) and the row's weights are staged too.
constexpr unsigned char kMaskedOut = 255;

template <typename T, int Q>
struct FwdRowsCfg {
    using G = TeamGeom<T, Q>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    static constexpr int TPB = TEAM >= 256 ? 1 : 256 / TEAM;
    static constexpr int THREADS = TPB * TEAM;
    static constexpr int REGION = (int)(Q * sizeof(cpx<T>)) > G::SCRATCH ? (int)(Q * sizeof(cpx<T>)) : G::SCRATCH;
    static constexpr size_t smem(int W, bool weighted) {
        return (size_t)TPB * REGION + (((size_t)W + 15) & ~(size_t)15) + (weighted ? (size_t)W * sizeof(double) : 0);
    }
};

template <typename T, int Q>
__global__ void __launch_bounds__(FwdRowsCfg<T, Q>::THREADS)
k_fwd_rows(const int32_t* __restrict__ X, const uint8_t* __restrict__ MX, const double* __restrict__ WX, int H, int W,
           int K, int Qs, cpx<T>* __restrict__ T1, Tw<T> tw, DevStatus* __restrict__ st, int conditional,
           int* __restrict__ popc, const unsigned char* __restrict__ plane_need) {
    // popc (nullable): per-label pixel counts under mask 1 are added to popc[0 .. K).
    // plane_need (nullable): only planes whose entry is 1 are transformed (a team
    // whose two planes are both unneeded idles; a block with no needed plane returns).
    using C = FwdRowsCfg<T, Q>;
    if (conditional && !(st->flags & STATUS_ESCALATE)) return;
    constexpr int M = C::M, R = C::R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* code = smem_raw + (size_t)C::TPB * C::REGION;
    double* wts = reinterpret_cast<double*>(code + (((size_t)W + 15) & ~(size_t)15));
    const int team = threadIdx.x / C::TEAM, lt = threadIdx.x % C::TEAM, r = lt / M, j = lt % M;
    const int npp = (K + 1) / 2;
    const int y = blockIdx.x, pp = blockIdx.y * C::TPB + team;
    auto needed = [&](int q) {
        if (q >= npp) return false;
        if (!plane_need) return true;
        return plane_need[2 * q] == 1 || (2 * q + 1 < K && plane_need[2 * q + 1] == 1);
    };
    if (plane_need) {
        bool any = false;
        for (int t = 0; t < C::TPB; ++t) any |= needed(blockIdx.y * C::TPB + t);
        if (!any) return;  // uniform over the block
    }
    const bool active = needed(pp);
    const int la = 2 * pp, lb = 2 * pp + 1;
    const int32_t* xr = X + (size_t)y * W;
    const uint8_t* mr = MX ? MX + (size_t)y * W : nullptr;
    bool bad = false;
    // weighted maps run with FP64 transforms only: the other precisions never read weights
    const double* wr = std::is_same<T, double>::value && WX ? WX + (size_t)y * W : nullptr;
    for (int x = threadIdx.x; x < W; x += C::THREADS) {
        const int lab = __ldg(xr + x);
        bool m = mr ? (__ldg(mr + x) != 0) : true;
        if (wr) {
            const double w = __ldg(wr + x);
            m = w > 0.0;
            wts[x] = w;
        }
        if (m && (lab < 0 || lab >= K)) bad = true;
        code[x] = m && lab >= 0 && lab < K ? (unsigned char)lab : kMaskedOut;
    }
    if (bad && blockIdx.y == 0) atomicOr(&st->flags, STATUS_LABEL_RANGE);
    __syncthreads();
    if (popc && blockIdx.y == 0) {
        // label histogram of the row (shared-memory bins in the first team's region,
        // which the transform below only overwrites after the next barrier)
        int* hist = reinterpret_cast<int*>(smem_raw);
        for (int k = threadIdx.x; k < K; k += C::THREADS) hist[k] = 0;
        __syncthreads();
        for (int x = threadIdx.x; x < W; x += C::THREADS) {
            const int c = code[x];
            if (c != kMaskedOut) atomicAdd(&hist[c], 1);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += C::THREADS)
            if (hist[k]) atomicAdd(&popc[k], hist[k]);
        __syncthreads();
    }
    unsigned char* region = smem_raw + (size_t)team * C::REGION;
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(region);
    auto load = [&](int x) -> cpx<T> {
        if (!active || x >= W) return {T(0), T(0)};
        const int c = code[x];
        T one = T(1);
        if constexpr (std::is_same<T, double>::value) {
            if (wr) one = wts[x];
        }
        return {c == la ? one : T(0), c == lb ? one : T(0)};
    };
    cpx<T> v[M];
    team_fft<M, R, -1>(v, r, j, load, region + r * grp_scratch_bytes<T, M>(), tw.sq[ilog2c(M)], tw_of<Q>(tw));
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) sm[R * (j + M * k2) + r] = v[brev(k2, M)];
    __syncthreads();
    if (!active) return;
    const T h = T(0.5);
    for (int k = lt; k <= Q / 2; k += C::TEAM) {
        const cpx<T> a = sm[k], b = sm[k == 0 ? 0 : Q - k];
        // F_la = (X[k] + conj X[-k]) / 2,  F_lb = (X[k] - conj X[-k]) / (2i)
        T1[((size_t)la * H + y) * Qs + k] = {h * (a.x + b.x), h * (a.y - b.y)};
        if (lb < K) T1[((size_t)lb * H + y) * Qs + k] = {h * (a.y + b.y), h * (b.x - a.x)};
    }
}

// ---------------------------------------------------------------------------
// Forward column transforms.  Block = (TPB adjacent kx columns, plane).  The
// block first stages its H x TPB input tile in shared memory with coalesced
// 16-byte loads (column slots XOR-swizzled by row, so that the teams' column
// reads are conflict-free), then each team transforms one column.
template <typename T, int P, int MMAX = max_m<T>()>
struct ColCfg {
    using G = TeamGeom<T, P, MMAX>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    static constexpr int TPB = TEAM >= 256 ? 1 : pow2_floor(256 / TEAM);  // a power of two (swizzle)
    static constexpr int THREADS = TPB * TEAM;
    static constexpr int SWZ = TPB >= 16 ? 0 : (TPB == 8 ? 1 : (TPB == 4 ? 2 : 3));
    static constexpr size_t SCR = (size_t)TPB * G::SCRATCH;
    static constexpr size_t TILE_MAX = (size_t)P * TPB * sizeof(cpx<T>);  // H <= P rows
    static constexpr size_t smem(int H) { return SCR + (size_t)H * TPB * sizeof(cpx<T>); }
};

template <typename T, int P, int MMAX>
__global__ void __launch_bounds__(ColCfg<T, P, MMAX>::THREADS, sizeof(T) == 4 && ColCfg<T, P, MMAX>::THREADS <= 256 ? 3 : 1)
k_fwd_cols(const cpx<T>* __restrict__ T1, int H, int nplanes, int Qh, int Qs, cpx<T>* __restrict__ F, Tw<T> tw,
           const DevStatus* __restrict__ st, int conditional, T out_scale,
           const unsigned char* __restrict__ plane_need, int slices) {
    // plane_need (nullable): only the planes of labels whose entry is 1 are
    // transformed; plane p belongs to label p / slices (volumes: slices = depth).
    using C = ColCfg<T, P, MMAX>;
    if (conditional && !(st->flags & STATUS_ESCALATE)) return;
    if (plane_need && plane_need[blockIdx.y / slices] != 1) return;
    constexpr int M = C::M, R = C::R, TPB = C::TPB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<T>* tile = reinterpret_cast<cpx<T>*>(smem_raw + C::SCR);
    const int team = threadIdx.x / C::TEAM, lt = threadIdx.x % C::TEAM, r = lt / M, j = lt % M;
    const int kx0 = blockIdx.x * TPB, kx = kx0 + team, plane = blockIdx.y;
    const cpx<T>* src = T1 + (size_t)plane * H * Qs + kx0;
    if constexpr (sizeof(T) == 4 && TPB >= 2) {
        // 16-byte pieces (two columns each); Qs and kx0 are even, so a piece is
        // wholly inside the row or wholly beyond Qs (never read: zeros)
        constexpr int PPR = TPB / 2;
        for (int q = threadIdx.x; q < H * PPR; q += C::THREADS) {
            const int y = q / PPR, h = q % PPR;
            float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kx0 + 2 * h < Qs) pv = __ldg(reinterpret_cast<const float4*>(src + (size_t)y * Qs) + h);
            const int sw = (y >> C::SWZ) & (TPB - 1);
            if (sw & 1) pv = make_float4(pv.z, pv.w, pv.x, pv.y);
            reinterpret_cast<float4*>(tile)[y * PPR + (h ^ (sw >> 1))] = pv;
        }
    } else {
        for (int q = threadIdx.x; q < H * TPB; q += C::THREADS) {
            const int y = q / TPB, c = q % TPB;
            const int sw = (y >> C::SWZ) & (TPB - 1);
            tile[y * TPB + (c ^ sw)] = kx0 + c < Qs ? src[(size_t)y * Qs + c] : cpx<T>{T(0), T(0)};
        }
    }
    __syncthreads();
    const bool active = kx < Qh;
    auto load = [&](int y) -> cpx<T> {
        if (!active || y >= H) return {T(0), T(0)};
        return tile[y * TPB + (team ^ ((y >> C::SWZ) & (TPB - 1)))];
    };
    cpx<T> v[M];
    team_fft<M, R, -1>(v, r, j, load, smem_raw + (size_t)team * C::G::SCRATCH + r * grp_scratch_bytes<T, M>(),
                       tw.sq[ilog2c(M)], tw_of<P>(tw));
    if (!active) return;
    // Column ky is stored at slot (ky % R) * M*M + ky / R: the samples that one
    // group of the pair-product transform (same P, same R) takes are contiguous.
    cpx<T>* out = F + ((size_t)plane * Qh + kx) * P;
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) {
        const cpx<T> z = v[brev(k2, M)];
        out[r * (M * M) + j + M * k2] = {z.x * out_scale, z.y * out_scale};
    }
}

// Read-only loads of complex values through the non-coherent path.
__device__ __forceinline__ cpx<float> __ldg(const cpx<float>* p) {
    const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> __ldg(const cpx<double>* p) {
    const double2 v = ::__ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<df32> __ldg(const cpx<df32>* p) {
    const float4 v = ::__ldg(reinterpret_cast<const float4*>(p));
    return {df32(v.x, v.y), df32(v.z, v.w)};
}

// ---------------------------------------------------------------------------
// Copy n twiddles from global to shared memory (whole block).
template <typename T>
__device__ __forceinline__ void stage_table(cpx<T>* dst, const cpx<T>* __restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Configuration of the pair-product + inverse column kernel (k_pair_cols below):
// TPB columns per block, one team of R x M lanes per column; the block's shared
// memory holds one buffer (the teams' exchange, then the P x TPB output tile,
// with the transpose scratch aliased on it) and the twiddle tables.
template <typename T, int P, int MMAX = max_m<T>()>
struct PairColsCfg {
    using G = TeamGeom<T, P, MMAX>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM, NQ = M * M;
    // at least 256 threads, and at least 32 bytes of adjacent kx per tile row (whole sectors)
    static constexpr int TPB0 = TEAM >= 256 ? 1 : pow2_floor(256 / TEAM);  // a power of two (swizzle)
    static constexpr int TPB = TPB0 * (int)sizeof(cpx<T>) >= 32 ? TPB0 : 32 / (int)sizeof(cpx<T>);
    static constexpr int THREADS = TPB * TEAM;
    static constexpr int PER = R > 2 ? M / R : 1;  // points per lane of the radix-R combine (R a power of two)
    static constexpr int PTS = (NQ + TEAM - 1) / TEAM;  // points per lane of the radix-3/6 combine
    static constexpr int SWZ = TPB >= 16 ? 0 : (TPB == 8 ? 1 : (TPB == 4 ? 2 : 3));
    // one buffer per block: the teams' group-transform exchange, then the P x TPB output tile
    static constexpr size_t XBUF = (size_t)TPB * P * sizeof(cpx<T>);
    static constexpr size_t FFT = (size_t)TPB * G::SCRATCH;
    static constexpr size_t MAIN = (XBUF > FFT ? XBUF : FFT);
    static constexpr size_t FFT_WIDE = (size_t)TPB * R * M * M * sizeof(cpx<T>);  // complex transposes
    static constexpr int TW_N = R == 2 ? P / 2 : (R > 2 ? P : 0);  // combine twiddles W_P^k
    static constexpr size_t SMEM = MAIN + (size_t)(NQ + TW_N) * sizeof(cpx<T>);
    // FP32: two blocks per SM (M = 32 needs 128 registers a thread, so 256 threads)
    static constexpr int MIN_BLOCKS = sizeof(T) == 4 && (M < 32 ? is_pow2(R) && THREADS <= 512 : THREADS <= 256) ? 2 : 1;
};

// Pair product + inverse column transform of length P = R*M*M.  Persistent
// blocks walk the items (pair, kx block) with pairs varying fastest, so that
// the items in flight at one time read the same few spectrum columns (L2
// reuse).  Decimation in time across the R groups of a team: group r
// transforms the M*M samples ky = R*m + r (every input is loaded and
// multiplied once per team), the groups exchange their sub-transforms through
// shared memory, and group r forms the outputs [r*M*M, (r+1)*M*M) by the
// radix-R butterfly (FP32 groups of 16 or 32 lanes transpose complex values in
// one pass through their M*M slice of the same buffer).  The exchange buffer then serves as a P x TPB tile
// (column slots XOR-swizzled by row, conflict-free writes) whose rows leave
// as chunks of TPB adjacent kx.  While the tile leaves, the F_a loads of the
// block's next item are already in flight, and items at the head of a kx
// block ask L2 for the spectrum columns two kx blocks ahead.  work_ctr must
// be zero at launch.
// VOL (volumes): items are (pair, depth offset dz, kx block); the product is
// the sum over the slices z of conj(F_a,z) F_b,z+dz (the 3-D correlation's
// depth sum, taken before the inverse transform, which is linear), and the
// output row of depth offset index dzo is dzo * R2 + (the image's output row).
template <typename T, int P, bool VOL, int MMAX>
__global__ void __launch_bounds__(PairColsCfg<T, P, MMAX>::THREADS, PairColsCfg<T, P, MMAX>::MIN_BLOCKS)
k_pair_cols(const cpx<T>* __restrict__ FA, const cpx<T>* __restrict__ FB, int KA, int KB, int Qh, int HA, int HB,
            int Rout, int Qs, int r0, int r1, cpx<T>* __restrict__ Y, Tw<T> tw, const DevStatus* __restrict__ st,
            int conditional, int* __restrict__ work_ctr, int DA, int DB, int R2, const int* __restrict__ plist,
            const int* __restrict__ lrange, int chunk_off, int chunk_cap, int units) {
    // units > 1 (images only): several floating images (rotation angles) at once;
    // unit u's spectra are F_b plane b * units + u, its output rows u * R2 + (row).
    // List mode (plist non-null): only the pairs plist[lrange[0] + chunk_off + e],
    // e < min(chunk_cap, lrange[1] - lrange[0] - chunk_off), are computed, pair e's
    // rows going to Y + e * Rout * Qs.
    using C = PairColsCfg<T, P, MMAX>;
    if (conditional && !(st->flags & STATUS_ESCALATE)) return;
    constexpr int M = C::M, R = C::R, TPB = C::TPB, NQ = C::NQ;
    const int Dz = VOL ? DA + DB - 1 : 1;
    int npairs = KA * KB, lbase = 0;
    if (plist) {
        lbase = lrange[0] + chunk_off;
        npairs = min(lrange[1] - lbase, chunk_cap);
        if (npairs <= 0) return;  // uniform: nothing listed for this launch
    }
    auto real_pair = [&](int e) { return plist ? ::__ldg(plist + lbase + e) : e; };
    const int U = VOL ? Dz : units;  // the middle item dimension: depth offsets or units
    const int nkxb = (Qh + TPB - 1) / TPB, n_items = npairs * nkxb * U;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    cpx<T>* xbuf = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* tw_sq = reinterpret_cast<cpx<T>*>(smem_raw + C::MAIN);
    cpx<T>* tw_n = tw_sq + NQ;
    // Items are handed out in order from a counter (zeroed before the launch), so
    // that the items in flight stay within a few kx blocks whatever the blocks' pace.
    if (threadIdx.x == 0) s_item = atomicAdd(work_ctr, 1);
    stage_table(tw_sq, tw.sq[ilog2c(M)], NQ);
    if (R > 1) stage_table(tw_n, tw_of<P>(tw), C::TW_N);
    __syncthreads();
    int item = s_item;
    if (item >= n_items) return;
    const int team = threadIdx.x / C::TEAM, lt = threadIdx.x % C::TEAM, r = lt / M, j = lt % M;
    // group r: the samples ky = R*m + r, m = j + M*i, stored contiguously from slot
    // r*NQ (the forward column transform's output order).  conj(F_a) F_b, F_b
    // carrying the 1/(P Q) of the inverse.
    cpx<T> v[M];
    cpx<T> wo[(R > 2 && !is_pow2(R)) ? C::PTS * R : 1];  // outputs of the radix-3/6 combine
    auto load_fa = [&](int it) {
        if constexpr (VOL) return;  // volumes sum over slices in the item itself
        const int kx = (VOL ? it / npairs / U : (it / npairs) % nkxb) * TPB + team, a = real_pair(it % npairs) / KB;
        if (kx < Qh) {
            const cpx<T>* ga = FA + ((size_t)a * Qh + kx) * P + r * NQ + j;
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = __ldg(ga + M * i);
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = {T(0), T(0)};
        }
    };
    load_fa(item);
    while (true) {
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(work_ctr, 1);
        const int e = item % npairs, pair = real_pair(e);
        // volumes: kx block outermost, then the depth offset (the slices' spectra of one
        // kx block serve every depth offset); units: the unit outermost, so that the
        // items in flight write the rows of few maps and complete their lines in L2
        const int kxb = VOL ? item / npairs / U : (item / npairs) % nkxb;
        const int dzo = VOL ? (item / npairs) % U : item / npairs / nkxb;  // VOL: depth offset index; else the unit
        const int kx0 = kxb * TPB, kx = kx0 + team, b = pair % KB;
        if constexpr (VOL) {
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = {T(0), T(0)};
            if (kx < Qh) {
                const int a = pair / KB, dz = dzo - (DA - 1);
                const int z0 = dz < 0 ? -dz : 0, z1 = DA < DB - dz ? DA : DB - dz;
                for (int z = z0; z < z1; ++z) {
                    const cpx<T>* ga = FA + ((size_t)(a * DA + z) * Qh + kx) * P + r * NQ + j;
                    const cpx<T>* gb = FB + ((size_t)(b * DB + z + dz) * Qh + kx) * P + r * NQ + j;
#pragma unroll
                    for (int i = 0; i < M; ++i) v[i] = v[i] + cmulc(__ldg(gb + M * i), __ldg(ga + M * i));
                }
            }
        } else if (kx < Qh) {
            const cpx<T>* gb = FB + ((size_t)(b * units + dzo) * Qh + kx) * P + r * NQ + j;
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = cmulc(__ldg(gb + M * i), v[i]);
        }
        if (!VOL && !plist && pair < KA + KB && (int)threadIdx.x < TPB && kxb + 2 < nkxb) {
            // the items of this kx block with pair < K_A + K_B each prefetch one
            // spectrum's columns of kx block kxb + 2 into L2 (one bulk request per column)
            const int kf = (kxb + 2) * TPB + threadIdx.x;
            if (kf < Qh) {
                const cpx<T>* src = pair < KA ? FA + ((size_t)pair * Qh + kf) * P
                                              : FB + ((size_t)((pair - KA) * units + dzo) * Qh + kf) * P;
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((unsigned)(P * sizeof(cpx<T>)))
                             : "memory");
            }
        }
        if constexpr (sizeof(T) == 4 && M >= 16 && C::FFT_WIDE <= C::MAIN)  // scratch of M*M complex per group
            // radix-2^2 register DFTs at R = 1 (at R = 2 both made the kernel spill, the
            // second alone measured no faster)
            team_fft_core<M, +1, true, true, R == 1 ? 3 : 0>(v, j, smem_raw + (size_t)(team * R + r) * (M * M * sizeof(cpx<T>)), tw_sq);
        else
            team_fft_core<M, +1>(v, j, smem_raw + (size_t)team * C::G::SCRATCH + r * grp_scratch_bytes<T, M>(), tw_sq);
        if (threadIdx.x == 0) s_item = next;  // read by all after the tile barrier below
        cpx<T>* tx = xbuf + (size_t)team * P;  // this team's R sub-transforms
        if constexpr (R == 2) {
            // X[k] = E_0[k] + W^k E_1[k], X[k + NQ] = E_0[k] - W^k E_1[k] (W = W_P, inverse
            // direction, W^NQ = -1).  Lane j of both groups holds the same k = j + M k2:
            // group 1 forms W^k E_1[k] once, the groups swap values through shared memory.
            __syncthreads();  // every group is done with its transpose scratch (aliases xbuf)
            if (r == 1) {
#pragma unroll
                for (int k2 = 0; k2 < M; ++k2)
                    v[brev(k2, M)] = cmul(v[brev(k2, M)], twl<+1>(tw_n, j + M * k2));
            }
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) tx[r * NQ + j + M * k2] = v[brev(k2, M)];
            __syncthreads();
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int k = j + M * k2;
                v[brev(k2, M)] = r == 0 ? v[brev(k2, M)] + tx[NQ + k] : tx[k] - v[brev(k2, M)];
            }
        } else if constexpr (R > 2 && !is_pow2(R)) {
            // R = 3, 6: as below, with the team's lanes l = r M + j taking the points
            // k = l + TEAM t (the outputs stay in wo[] until the exchange reads are done)
            __syncthreads();  // every group is done with its transpose scratch (aliases xbuf)
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int k = j + M * k2;
                const cpx<T> e = v[brev(k2, M)];
                tx[r * NQ + k] = r ? cmul(e, twl<+1>(tw_n, r * k)) : e;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < C::PTS; ++t) {
                const int k = lt + C::TEAM * t;
                if (C::PTS * C::TEAM == NQ || k < NQ) {
                    cpx<T> u[R];
#pragma unroll
                    for (int s2 = 0; s2 < R; ++s2) u[s2] = tx[s2 * NQ + k];
                    dft_nat<R, +1>(u);
#pragma unroll
                    for (int q = 0; q < R; ++q) wo[t * R + q] = u[q];
                }
            }
        } else if constexpr (R > 2) {
            // X[k + q NQ] = sum_s w_R^{sq} (W^{sk} E_s[k]) (W = W_P, inverse direction): group
            // s twiddles its own values, the team exchanges them through shared memory, and
            // lane (r, j) forms all R outputs of the points k = j + M (r PER + t), t < PER,
            // with an R-point DFT in registers (outputs kept as v[t R + q]).
            __syncthreads();  // every group is done with its transpose scratch (aliases xbuf)
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int k = j + M * k2;
                const cpx<T> e = v[brev(k2, M)];
                tx[r * NQ + k] = r ? cmul(e, twl<+1>(tw_n, r * k)) : e;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < C::PER; ++t) {
                const int k = j + M * (r * C::PER + t);
                cpx<T> u[R];
#pragma unroll
                for (int s2 = 0; s2 < R; ++s2) u[s2] = tx[s2 * NQ + k];
                dft_reg<R, +1>(u);
#pragma unroll
                for (int q = 0; q < R; ++q) v[t * R + q] = u[brev(q, R)];
            }
        }
        __syncthreads();  // exchange reads done: the buffer becomes the tile
        // tile slot (row, team) swizzled by row
        if constexpr (R > 2 && !is_pow2(R)) {
#pragma unroll
            for (int t = 0; t < C::PTS; ++t) {
                const int k = lt + C::TEAM * t;
                if (C::PTS * C::TEAM == NQ || k < NQ) {
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int row = k + q * NQ;
                        xbuf[(size_t)row * TPB + (team ^ ((row >> C::SWZ) & (TPB - 1)))] = wo[t * R + q];
                    }
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                int row;
                cpx<T> val;
                if constexpr (R > 2) {
                    row = j + M * (r * C::PER + i / R) + (i % R) * NQ;
                    val = v[i];
                } else {
                    row = r * NQ + j + M * i;
                    val = v[brev(i, M)];
                }
                xbuf[(size_t)row * TPB + (team ^ ((row >> C::SWZ) & (TPB - 1)))] = val;
            }
        }
        __syncthreads();
        next = s_item;
        if (next < n_items) load_fa(next);
        cpx<T>* yp = Y + (size_t)e * Rout * Qs;
        if constexpr (sizeof(T) == 4 && TPB >= 2) {
            // Each row chunk of TPB complex leaves as TPB/2 16-byte pieces written by
            // adjacent lanes.  Logical columns 2h, 2h+1 sit in physical piece
            // h ^ (sw >> 1), swapped when sw is odd.  Qs and kx0 are even, so a
            // piece is either wholly inside the row (kx0 + 2h < Qs) or wholly out;
            // for TPB <= 4 always inside (Qs is a multiple of 4).
            constexpr int PPR = TPB / 2, ROWS = C::THREADS / PPR;
            if constexpr (ROWS % (TPB << C::SWZ) == 0) {
                // A thread keeps its piece h and visits rows row0 + i * ROWS; ROWS is a
                // multiple of the swizzle period, so the swizzle is fixed per thread.
                const int h = threadIdx.x % PPR, row0 = threadIdx.x / PPR;
                const int sw = (row0 >> C::SWZ) & (TPB - 1);
                const bool swap_halves = sw & 1;
                if (TPB <= 4 || kx0 + 2 * h < Qs) {
                    const float4* src = reinterpret_cast<const float4*>(xbuf) + row0 * PPR + (h ^ (sw >> 1));
                    float4* dst = reinterpret_cast<float4*>(yp + kx0) + h;
                    for (int row = row0; row < P; row += ROWS, src += ROWS * PPR) {
                        int orow = circ_to_out(row, P, HA, HB - 1);
                        if constexpr (VOL) {
                            if (orow < 0) continue;
                            orow += dzo * R2;
                        }
                        if (orow < r0 || orow >= r1) continue;
                        if constexpr (!VOL) orow += dzo * R2;  // the unit's rows
                        float4 pv = *src;
                        if (swap_halves) pv = make_float4(pv.z, pv.w, pv.x, pv.y);
                        dst[(size_t)orow * (Qs / 2)] = pv;
                    }
                }
            } else {
                for (int q = threadIdx.x; q < P * PPR; q += C::THREADS) {
                    const int row = q / PPR, h = q % PPR;
                    int orow = circ_to_out(row, P, HA, HB - 1);
                    if constexpr (VOL) {
                        if (orow < 0) continue;
                        orow += dzo * R2;
                    }
                    if (orow < r0 || orow >= r1 || kx0 + 2 * h >= Qs) continue;
                    if constexpr (!VOL) orow += dzo * R2;
                    const int sw = (row >> C::SWZ) & (TPB - 1);
                    float4 pv = reinterpret_cast<const float4*>(xbuf)[row * PPR + (h ^ (sw >> 1))];
                    if (sw & 1) pv = make_float4(pv.z, pv.w, pv.x, pv.y);
                    reinterpret_cast<float4*>(yp + (size_t)orow * Qs + kx0)[h] = pv;
                }
            }
        } else {
            // one complex per lane, adjacent lanes on adjacent columns of a row
            for (int q = threadIdx.x; q < P * TPB; q += C::THREADS) {
                const int row = q / TPB, c = q % TPB;
                int orow = circ_to_out(row, P, HA, HB - 1);
                if constexpr (VOL) {
                    if (orow < 0) continue;
                    orow += dzo * R2;
                }
                if (orow < r0 || orow >= r1 || kx0 + c >= Qs) continue;
                if constexpr (!VOL) orow += dzo * R2;
                const int sw = (row >> C::SWZ) & (TPB - 1);
                yp[(size_t)orow * Qs + kx0 + c] = xbuf[(size_t)row * TPB + (c ^ sw)];
            }
        }
        __syncthreads();  // tile reads (and s_item) done before the next item reuses them
        if (next >= n_items) break;
        item = next;
    }
}

template <typename T, int P, int MMAX = max_m<T>()>
constexpr size_t pair_cols_smem() {
    return PairColsCfg<T, P, MMAX>::SMEM;
}

// ---------------------------------------------------------------------------
// Inverse row transform (complex-to-real, length Q) + fused entropy epilogue.
// One block per output row (grid-stride).  Per round, NT teams transform NT
// pairs (a-major order); each thread then owns fixed shift positions p and
// accumulates, pair by pair, the joint term T(c), the running A-marginal of
// the current label a, and the B-marginal C_B^b(p) (shared or global memory).
// The rounded counts reach the owners through the teams' scratch, in HALVES
// passes (two for FP32, whose scratch holds half a row).
template <typename T, int Q>
struct RowCfg {
    static constexpr int L = Q / 2;
    using G = TeamGeom<T, L>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    // FP32: one thread per position of a pass (Q / 2), between one warp and 512
    // threads, so that no thread idles in the epilogue; smaller blocks share an SM.
    static constexpr int BT_TARGET = sizeof(T) == 4 ? (Q / 2 >= 512 ? 512 : (Q / 2 >= 32 ? Q / 2 : 32)) : 256;
    // FP32: as many teams as the target allows, fewer when that lets the threads divide
    // a pass's positions exactly (no idle lanes in the epilogue) at no more than a
    // quarter fewer teams (3072: 4 teams of 96 lanes, 1536: 8 of 48)
    static constexpr int NT0 = TEAM >= BT_TARGET ? 1 : BT_TARGET / TEAM;
    static constexpr int nt_exact(int nt) {
        return nt <= 1 ? 1 : ((Q / (sizeof(T) == 4 ? 2 : 1)) % (nt * TEAM) == 0 ? nt : nt_exact(nt - 1));
    }
    static constexpr int NT = (sizeof(T) == 4 && nt_exact(NT0) * 4 >= NT0 * 3) ? nt_exact(NT0) : NT0;
    static constexpr int THREADS = NT * TEAM;
    static constexpr int HALVES = sizeof(T) == 4 ? 2 : 1;
    static constexpr int QH = Q / HALVES;                      // positions per pass
    static constexpr int UH = (QH + THREADS - 1) / THREADS;    // positions per thread per pass
    static constexpr int U = HALVES * UH;
    static constexpr int REGION = G::SCRATCH;                  // >= QH floats
    static constexpr size_t TEAM_SMEM = (size_t)NT * REGION;
    // FP32: each team's next Y row (L + 1 complex, 16-byte chunks) is copied into a
    // shared-memory buffer by asynchronous copies (cp.async) while the current round
    // computes; the transform then loads its inputs from shared memory
    static constexpr bool STAGE = sizeof(T) == 4;
    static constexpr int STAGE_BYTES = STAGE ? ((L + 1) * 8 + 15) / 16 * 16 : 0;
    static constexpr size_t OFF_STAGE = (TEAM_SMEM + 15) / 16 * 16;
    static constexpr size_t OFF_CB = OFF_STAGE + (size_t)NT * STAGE_BYTES;  // B-marginals (shared-memory variant)
    static constexpr int MIN_BLOCKS = sizeof(T) == 4 && THREADS < 512 ? 512 / THREADS : 1;  // <= 128 registers
    static_assert(REGION >= QH * 4, "team scratch must hold one pass of rounded counts");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// 16-byte asynchronous global-to-shared copy (L2 only), its group commit and the
// wait for all of this thread's copies
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, int Q, bool CB_SMEM, bool NMI>
__global__ void __launch_bounds__(RowCfg<T, Q>::THREADS, RowCfg<T, Q>::MIN_BLOCKS)
k_pair_rows(const cpx<T>* __restrict__ Y, Geom g, Tw<T> tw, float* __restrict__ cb_global,
            double* __restrict__ mi_map, int32_t* __restrict__ n_map, int32_t* __restrict__ counts,
            DevStatus* __restrict__ st, int prec_slot, int conditional, const int32_t* __restrict__ ov,
            const int* __restrict__ ov_slot, unsigned* __restrict__ pair_res) {
    // ov / ov_slot (nullable): a pair with ov_slot[pair] = s >= 0 takes its counts
    // from ov[s][row][position] (exact counts from the second precision) instead of
    // its own transform, and its residual is not counted.  pair_res (nullable):
    // each pair's largest residual is folded into pair_res[pair].
    using C = RowCfg<T, Q>;
    constexpr int M = C::M, R = C::R, L = C::L, NT = C::NT, U = C::U, UH = C::UH, BT = C::THREADS;
    constexpr int HALVES = C::HALVES, QH = C::QH;
    if (conditional && !(st->flags & STATUS_ESCALATE)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* cb = CB_SMEM ? reinterpret_cast<float*>(smem_raw + C::OFF_CB)
                        : cb_global + (size_t)blockIdx.x * g.KB * Q;
    const int tid = threadIdx.x, team = tid / C::TEAM, lt = tid % C::TEAM, r = lt / M, j = lt % M;
    unsigned char* region = smem_raw + (size_t)team * C::REGION;
    const int KA = g.KA, KB = g.KB, npairs = KA * KB, Rout = g.R, Cout = g.C, Qs = g.Qs;
    const size_t RC = (size_t)Rout * Cout;
    const cpx<T>* twq_c2r = tw_of<Q>(tw);
    float res_max = 0.f;
    int row_max_n = 0;

    // tasks: the window's rows of every unit (units > 1: several maps, R2 rows apart)
    const int nr = g.r1 - g.r0, ntask = g.units * nr;
    auto task_row = [&](int tk) { return (tk / nr) * g.R2 + g.r0 + tk % nr; };
    // STAGE: the team's buffer for the Y row of its current pair; the team's lanes
    // copy a row in 16-byte chunks (the rows start on 32-byte boundaries: Qs is a
    // multiple of 4 complex)
    const cpx<T>* stage = reinterpret_cast<const cpx<T>*>(smem_raw + C::OFF_STAGE + (size_t)team * C::STAGE_BYTES);
    auto stage_issue = [&](int pair_i, int row_i) {
        if constexpr (C::STAGE) {
            const char* src = reinterpret_cast<const char*>(Y + ((size_t)pair_i * Rout + row_i) * Qs);
            const uint32_t dst = smem_u32(stage);
            for (int c = lt; c < C::STAGE_BYTES / 16; c += C::TEAM) cp_async16(dst + 16u * c, src + 16 * c);
            cp_async_commit();
        }
    };
    if constexpr (C::STAGE) {
        if ((int)blockIdx.x < ntask && team < npairs) stage_issue(team, task_row(blockIdx.x));
        cp_async_wait_all();
        __syncthreads();
    }
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int row = task_row(task);
        EntAcc<NMI> S[U];
        float CA[U];
        int N[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { S[u].zero(); CA[u] = 0.f; N[u] = 0; }
        for (int b = 0; b < KB; ++b)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pl = tid + BT * (u % UH), p = (u / UH) * QH + pl;
                if (pl < QH) cb[(size_t)b * Q + p] = 0.f;
            }
        int cur_a[HALVES];
#pragma unroll
        for (int hf = 0; hf < HALVES; ++hf) cur_a[hf] = 0;
        for (int base = 0; base < npairs; base += NT) {
            const int pair = base + team;
            const bool act = pair < npairs;
            const int ovs = (act && ov_slot) ? ov_slot[pair] : -1;
            const cpx<T>* yr = C::STAGE ? stage : Y + ((size_t)(act ? pair : 0) * Rout + row) * Qs;
            if (!C::STAGE && lt == 0) {
                // ask L2 for this team's row of the next round (or of the block's next row)
                int np = pair + NT, nrow = row;
                if (np >= npairs) {
                    np = team;
                    const int nt2 = task + (int)gridDim.x;
                    nrow = nt2 < ntask ? (nt2 / nr) * g.R2 + g.r0 + nt2 % nr : -1;
                }
                if (np < npairs && nrow >= 0)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Y + ((size_t)np * Rout + nrow) * Qs),
                                 "r"((unsigned)(Qs * sizeof(cpx<T>))) : "memory");
            }
            // Hermitian split: z = IDFT_L(E + iO), z[m] = x[2m] + i x[2m+1]
            auto load = [&](int k) -> cpx<T> {
                if (!act) return {T(0), T(0)};
                const cpx<T> yk = yr[k], ym = yr[L - k];
                const cpx<T> e = {yk.x + ym.x, yk.y - ym.y};
                const cpx<T> d = {yk.x - ym.x, yk.y + ym.y};
                const cpx<T> o = cmul(d, twl<+1>(twq_c2r, k));
                return {e.x - o.y, e.y + o.x};
            };
            cpx<T> v[M];
            team_fft<M, R, +1>(v, r, j, load, region + r * grp_scratch_bytes<T, M>(), tw.sq[ilog2c(M)],
                               tw_of<L>(tw));
            // round to the nearest integer; track the worst residual (the exactness guard)
            float rp = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const T cr = rint_t<T>(v[k].x), ci = rint_t<T>(v[k].y);
                rp = fmaxf(rp, fmaxf((float)fabs(v[k].x - cr), (float)fabs(v[k].y - ci)));
                v[k].x = cr;
                v[k].y = ci;
            }
            if (ovs < 0) res_max = fmaxf(res_max, rp);
            if (pair_res) {  // per-pair residual: reduce over the team's lanes of each warp
                constexpr int WID = C::TEAM < 32 ? C::TEAM : 32;
                float rr = (act && ovs < 0) ? rp : 0.f;
#pragma unroll
                for (int off = WID / 2; off > 0; off >>= 1) rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, off));
                if (act && ovs < 0 && (lt % WID) == 0) atomic_max_float_pos(&pair_res[pair], rr);
            }
            const int nt = min(NT, npairs - base);
            const int a0 = base / KB, b0 = base - a0 * KB;
#pragma unroll
            for (int hf = 0; hf < HALVES; ++hf) {
                __syncthreads();  // all scratch reads (FFT or previous pass) done
                if (C::STAGE && hf == 0) {
                    // the staged rows are consumed: copy this team's next row (the next
                    // round of this task, else round 0 of the block's next task)
                    int np = pair + NT, ntk = task;
                    if (np >= npairs) { np = team; ntk = task + (int)gridDim.x; }
                    if (np < npairs && ntk < ntask) stage_issue(np, task_row(ntk));
                }
                float2* ob = reinterpret_cast<float2*>(region);
#pragma unroll
                for (int k2 = hf * (M / HALVES); k2 < (hf + 1) * (M / HALVES); ++k2) {
                    const int mf = R * (j + M * k2) + r, m = mf - hf * (L / HALVES);
                    if (ovs >= 0) {  // exact counts of positions 2 mf, 2 mf + 1 from the second precision
                        const int2 q = *reinterpret_cast<const int2*>(ov + ((size_t)ovs * Rout + row) * Q + 2 * mf);
                        ob[m] = make_float2((float)q.x, (float)q.y);
                    } else {
                        const cpx<T> z = v[brev(k2, M)];
                        ob[m] = make_float2((float)z.x, (float)z.y);
                    }
                }
                __syncthreads();
                // the round's accumulation, compiled twice: with the debug count maps
                // and without (no per-count test of the counts pointer)
                auto accumulate = [&](auto dbg) {
                    constexpr bool DBG = decltype(dbg)::value;
                    int a = a0, b = b0;
                    if constexpr (!CB_SMEM && !DBG && NT * UH <= 16 && C::THREADS <= 384) {  // registers to spare
                        if (nt == NT && NT <= KB) {
                            // the round's pairs have distinct labels b: load their B-marginal
                            // slots (global memory) together, one memory latency per pass
                            // instead of one per pair
                            float cbv[NT][UH];
#pragma unroll
                            for (int t = 0; t < NT; ++t) {
                                const float* cbb = cb + (size_t)b * Q + hf * QH;
#pragma unroll
                                for (int uh = 0; uh < UH; ++uh) {
                                    const int pl = tid + BT * uh;
                                    cbv[t][uh] = pl < QH ? cbb[pl] : 0.f;
                                }
                                if (++b == KB) b = 0;
                            }
                            b = b0;
#pragma unroll
                            for (int t = 0; t < NT; ++t) {
                                if (a != cur_a[hf]) {
#pragma unroll
                                    for (int uh = 0; uh < UH; ++uh) {
                                        const int u = hf * UH + uh, pl = tid + BT * uh;
                                        if (pl >= QH) continue;
                                        S[u].marg(clog2c_fixed(CA[u]));
                                        N[u] += (int)CA[u];
                                        CA[u] = 0.f;
                                    }
                                    cur_a[hf] = a;
                                }
                                const float* obt = reinterpret_cast<const float*>(smem_raw + (size_t)t * C::REGION);
                                float* cbb = cb + (size_t)b * Q + hf * QH;
#pragma unroll
                                for (int uh = 0; uh < UH; ++uh) {
                                    const int u = hf * UH + uh, pl = tid + BT * uh;
                                    if (pl >= QH) continue;
                                    const float c = obt[pl];
                                    S[u].joint(clog2c_fixed(c));
                                    CA[u] += c;
                                    cbb[pl] = cbv[t][uh] + c;
                                }
                                if (++b == KB) { b = 0; ++a; }
                            }
                            return;
                        }
                    }
                    for (int t = 0; t < nt; ++t) {
                        if (a != cur_a[hf]) {  // uniform: the A-marginal of label cur_a is complete
#pragma unroll
                            for (int uh = 0; uh < UH; ++uh) {
                                const int u = hf * UH + uh, pl = tid + BT * uh;
                                if (pl >= QH) continue;
                                S[u].marg(clog2c_fixed(CA[u]));
                                N[u] += (int)CA[u];
                                if constexpr (DBG) {
                                    const int c = circ_to_out(hf * QH + pl, Q, g.WA, g.WB - 1);
                                    if (c >= 0)
                                        counts[((size_t)npairs + cur_a[hf]) * RC + (size_t)row * Cout + c] = (int)CA[u];
                                }
                                CA[u] = 0.f;
                            }
                            cur_a[hf] = a;
                        }
                        const float* obt = reinterpret_cast<const float*>(smem_raw + (size_t)t * C::REGION);
                        float* cbb = cb + (size_t)b * Q + hf * QH;
#pragma unroll
                        for (int uh = 0; uh < UH; ++uh) {
                            const int u = hf * UH + uh, pl = tid + BT * uh;
                            if (pl >= QH) continue;
                            const float c = obt[pl];
                            S[u].joint(clog2c_fixed(c));
                            CA[u] += c;
                            cbb[pl] += c;
                            if constexpr (DBG) {
                                const int cc = circ_to_out(hf * QH + pl, Q, g.WA, g.WB - 1);
                                if (cc >= 0) counts[(size_t)(base + t) * RC + (size_t)row * Cout + cc] = (int)c;
                            }
                        }
                        if (++b == KB) { b = 0; ++a; }
                    }
                };
                if (counts) accumulate(std::true_type{});
                else accumulate(std::false_type{});
            }
            if constexpr (C::STAGE) cp_async_wait_all();  // the next round's rows, visible after the barrier
            __syncthreads();  // the next round's transforms overwrite the scratch read above
        }
        // the B-marginals: all of this thread's positions of one label loaded together
        for (int b = 0; b < KB; ++b) {
            float cbv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pl = tid + BT * (u % UH), p = (u / UH) * QH + pl;
                cbv[u] = pl < QH ? cb[(size_t)b * Q + p] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pl = tid + BT * (u % UH), p = (u / UH) * QH + pl;
                if (pl >= QH) continue;
                S[u].marg(clog2c_fixed(cbv[u]));
                if (counts) {
                    const int cidx = circ_to_out(p, Q, g.WA, g.WB - 1);
                    if (cidx >= 0) counts[((size_t)npairs + KA + b) * RC + (size_t)row * Cout + cidx] = (int)cbv[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int pl = tid + BT * (u % UH), p = (u / UH) * QH + pl;
            if (pl >= QH) continue;
            const int cidx = circ_to_out(p, Q, g.WA, g.WB - 1);
            S[u].marg(clog2c_fixed(CA[u]));
            N[u] += (int)CA[u];
            if (counts && cidx >= 0) counts[((size_t)npairs + cur_a[u / UH]) * RC + (size_t)row * Cout + cidx] = (int)CA[u];
            if (cidx < 0) continue;
            const size_t o = (size_t)row * Cout + cidx;
            mi_map[o] = S[u].finish(N[u]);
            if (n_map) n_map[o] = N[u];
            if (cidx >= g.c0 && cidx < g.c1) row_max_n = max(row_max_n, N[u]);
        }
        __syncthreads();
    }
    // block reductions of the residual and max N
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        res_max = fmaxf(res_max, __shfl_xor_sync(0xffffffffu, res_max, off));
        row_max_n = max(row_max_n, __shfl_xor_sync(0xffffffffu, row_max_n, off));
    }
    if ((tid & 31) == 0) {
        atomic_max_float_pos(&st->res_bits[prec_slot], res_max);
        atomicMax(&st->max_n, row_max_n);
    }
}

// ---------------------------------------------------------------------------
// Exact counts of listed pairs in the second precision (per-pair escalation of
// CMIF_AUTO): the inverse row transform (complex-to-real, length Q) of rows
// [r0, r1) of the chunk's column-inverted products, rounded to the nearest
// integers (Sec. 3.2).  The counts of list slot s = lrange[0] + chunk_off + e
// (chunk pair e) go to ov[s][row][0 .. Q); the FP32 row kernels then take them
// in place of their own.  The largest residual goes to st->res_bits[1].
template <typename T, int Q>
struct RowCntCfg {
    static constexpr int L = Q / 2;
    using G = TeamGeom<T, L>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    static constexpr int NT = TEAM >= 128 ? 1 : 128 / TEAM;
    static constexpr int THREADS = NT * TEAM;
    static constexpr size_t SMEM = (size_t)NT * G::SCRATCH;
};

template <typename T, int Q>
__global__ void __launch_bounds__(RowCntCfg<T, Q>::THREADS)
k_pair_rows_counts(const cpx<T>* __restrict__ Y, Geom g, Tw<T> tw, const int* __restrict__ lrange, int chunk_off,
                   int chunk_cap, int32_t* __restrict__ ov, DevStatus* __restrict__ st) {
    using C = RowCntCfg<T, Q>;
    constexpr int M = C::M, R = C::R, L = C::L, NT = C::NT;
    const int lbase = lrange[0] + chunk_off;
    const int np = min(lrange[1] - lbase, chunk_cap);
    if (np <= 0) return;  // uniform: nothing listed for this launch
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int team = threadIdx.x / C::TEAM, lt = threadIdx.x % C::TEAM, r = lt / M, j = lt % M;
    unsigned char* region = smem_raw + (size_t)team * C::G::SCRATCH;
    const int nrows = g.r1 - g.r0;
    const long long ntask = (long long)np * nrows;
    const cpx<T>* twq_c2r = tw_of<Q>(tw);
    float res = 0.f;
    // a uniform trip count per block: every lane of a warp takes part in each transform's warp syncs
    for (long long t0 = (long long)blockIdx.x * NT; t0 < ntask; t0 += (long long)gridDim.x * NT) {
        const long long t = t0 + team;
        const bool act = t < ntask;
        const int e = act ? (int)(t / nrows) : 0, row = g.r0 + (act ? (int)(t % nrows) : 0);
        const cpx<T>* yr = Y + ((size_t)e * g.R + row) * g.Qs;
        // Hermitian split: z = IDFT_L(E + iO), z[m] = x[2m] + i x[2m+1]
        auto load = [&](int k) -> cpx<T> {
            if (!act) return {T(0), T(0)};
            const cpx<T> yk = yr[k], ym = yr[L - k];
            const cpx<T> ev = {yk.x + ym.x, yk.y - ym.y};
            const cpx<T> d = {yk.x - ym.x, yk.y + ym.y};
            const cpx<T> o = cmul(d, twl<+1>(twq_c2r, k));
            return {ev.x - o.y, ev.y + o.x};
        };
        cpx<T> v[M];
        team_fft<M, R, +1>(v, r, j, load, region + r * grp_scratch_bytes<T, M>(), tw.sq[ilog2c(M)],
                           tw_of<L>(tw));
        if (act) {
            int32_t* o = ov + ((size_t)(lbase + e) * g.R + row) * Q;
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const int mf = R * (j + M * k2) + r;
                const cpx<T> z = v[brev(k2, M)];
                const T cr = rint_t<T>(z.x), ci = rint_t<T>(z.y);
                res = fmaxf(res, fmaxf((float)fabs(z.x - cr), (float)fabs(z.y - ci)));
                *reinterpret_cast<int2*>(o + 2 * mf) = make_int2((int)(float)cr, (int)(float)ci);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) res = fmaxf(res, __shfl_xor_sync(0xffffffffu, res, off));
    if ((threadIdx.x & 31) == 0) atomic_max_float_pos(&st->res_bits[1], res);
}

// ---------------------------------------------------------------------------
// Spatially weighted MI (Sec. 3.3): the inverse row transform of weighted
// correlations (FP64 transforms) and the MI of their real-valued counts.  The
// counts are not integers, so nothing is rounded: each position accumulates
// sum c log2 c over joint, A- and B-marginal counts in FP64, with c log2 c = 0
// for c <= 0 (a count that the transform's rounding error takes below 0).
// MI = (S_joint - S_A - S_B + N log2 N) / N, N = sum_a C_A^a; 0 when N <= 0.
// One block per output row (grid-stride), NT teams transform NT pairs per round
// (a-major order); the B-marginals live in the block's global slice cbw.
template <int Q>
struct RowWCfg {
    static constexpr int L = Q / 2;
    using G = TeamGeom<double, L>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    static constexpr int NT = TEAM >= 256 ? 1 : 256 / TEAM;
    static constexpr int THREADS = NT * TEAM;
    static constexpr int U = (Q + THREADS - 1) / THREADS;  // positions per thread
    static constexpr int REGION = G::SCRATCH;              // one row of Q doubles
    static constexpr size_t SMEM = (size_t)NT * REGION;
    static_assert(REGION >= Q * 8, "team scratch must hold one row of counts");
};

__device__ __forceinline__ double xlog2x(double c) { return c > 0.0 ? c * log2(c) : 0.0; }

template <int Q>
__global__ void __launch_bounds__(RowWCfg<Q>::THREADS, 1)
k_pair_rows_w(const cpx<double>* __restrict__ Y, Geom g, Tw<double> tw, double* __restrict__ cbw,
              double* __restrict__ mi_map, double* __restrict__ nw_map, DevStatus* __restrict__ st) {
    using C = RowWCfg<Q>;
    constexpr int M = C::M, R = C::R, L = C::L, NT = C::NT, U = C::U, BT = C::THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, team = tid / C::TEAM, lt = tid % C::TEAM, r = lt / M, j = lt % M;
    unsigned char* region = smem_raw + (size_t)team * C::REGION;
    const int KB = g.KB, npairs = g.KA * g.KB, Rout = g.R, Cout = g.C, Qs = g.Qs;
    double* cb = cbw + (size_t)blockIdx.x * KB * Q;
    const cpx<double>* twq_c2r = tw_of<Q>(tw);
    double row_max_n = 0.0;
    for (int row = g.r0 + blockIdx.x; row < g.r1; row += gridDim.x) {
        double S[U], CA[U], N[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { S[u] = 0.0; CA[u] = 0.0; N[u] = 0.0; }
        for (int b = 0; b < KB; ++b)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = tid + BT * u;
                if (p < Q) cb[(size_t)b * Q + p] = 0.0;
            }
        int cur_a = 0;
        for (int base = 0; base < npairs; base += NT) {
            const int pair = base + team;
            const bool act = pair < npairs;
            const cpx<double>* yr = Y + ((size_t)(act ? pair : 0) * Rout + row) * Qs;
            // Hermitian split: z = IDFT_L(E + iO), z[m] = x[2m] + i x[2m+1]
            auto load = [&](int k) -> cpx<double> {
                if (!act) return {0.0, 0.0};
                const cpx<double> yk = yr[k], ym = yr[L - k];
                const cpx<double> e = {yk.x + ym.x, yk.y - ym.y};
                const cpx<double> d = {yk.x - ym.x, yk.y + ym.y};
                const cpx<double> o = cmul(d, twl<+1>(twq_c2r, k));
                return {e.x - o.y, e.y + o.x};
            };
            cpx<double> v[M];
            team_fft<M, R, +1>(v, r, j, load, region + r * grp_scratch_bytes<double, M>(), tw.sq[ilog2c(M)],
                               tw_of<L>(tw));
            __syncthreads();  // all transforms done with their scratch
            double2* ob = reinterpret_cast<double2*>(region);
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) {
                const cpx<double> z = v[brev(k2, M)];
                ob[R * (j + M * k2) + r] = make_double2(z.x, z.y);  // positions 2m, 2m + 1
            }
            __syncthreads();
            const int nt = min(NT, npairs - base);
            int a = base / KB, b = base - (base / KB) * KB;
            for (int t = 0; t < nt; ++t) {
                if (a != cur_a) {  // uniform: the A-marginal of label cur_a is complete
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        S[u] -= xlog2x(CA[u]);
                        N[u] += CA[u];
                        CA[u] = 0.0;
                    }
                    cur_a = a;
                }
                const double* obt = reinterpret_cast<const double*>(smem_raw + (size_t)t * C::REGION);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = tid + BT * u;
                    if (p >= Q) continue;
                    const double c = fmax(obt[p], 0.0);
                    S[u] += xlog2x(c);
                    CA[u] += c;
                    cb[(size_t)b * Q + p] += c;
                }
                if (++b == KB) { b = 0; ++a; }
            }
            __syncthreads();  // the next round's transforms overwrite the scratch read above
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = tid + BT * u;
            if (p >= Q) continue;
            S[u] -= xlog2x(CA[u]);
            N[u] += CA[u];
            for (int b = 0; b < KB; ++b) S[u] -= xlog2x(cb[(size_t)b * Q + p]);
            const int cidx = circ_to_out(p, Q, g.WA, g.WB - 1);
            if (cidx < 0) continue;
            const size_t o = (size_t)row * Cout + cidx;
            mi_map[o] = N[u] > 0.0 ? (S[u] + xlog2x(N[u])) / N[u] : 0.0;
            nw_map[o] = N[u];
            if (cidx >= g.c0 && cidx < g.c1) row_max_n = fmax(row_max_n, N[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) row_max_n = fmax(row_max_n, __shfl_xor_sync(0xffffffffu, row_max_n, off));
    if ((tid & 31) == 0) atomicMax(&st->max_nw_bits, (unsigned long long)__double_as_longlong(row_max_n));
}

template <typename T, int Q>
constexpr size_t pair_rows_smem(int KB, bool cb_smem) {
    return RowCfg<T, Q>::OFF_CB + (cb_smem ? (size_t)KB * Q * sizeof(float) : 0);
}

// ---------------------------------------------------------------------------
// gamma-gated argmax of Alg. 1 over one map: N_cal = gamma * max N; best MI
// among shifts with N >= N_cal; ties to the lowest map index.
struct PeakPart {
    double mi;
    long long idx;
};



}  // namespace cmif
