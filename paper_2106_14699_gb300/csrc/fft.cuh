// Register / shared-memory FFT building blocks for the CMIF transforms.
//
// The paper computes every cross-correlation of Eq. correlationjointhisto
// in the frequency domain with FFTs (Sec. 3.5, Eq. maincomplexity).  These
// are the transforms, written for sm_103a:
//
//  * dft_reg<M>     : an M-point DFT (M = 2..32) held in one thread's
//                     registers, radix-2 decimation in frequency, twiddles
//                     folded to compile-time constants (optionally in the
//                     radix-2^2 order, fewer general rotations).  Output in
//                     bit-reversed register order.
//  * team_fft<M,R>  : a length N = R*M*M DFT done by a "team" of R groups of
//                     M lanes (M points per lane).  The four-step split
//                     N' = M*M needs a single shared-memory transpose (XOR
//                     swizzled, conflict-free); R > 1 adds a radix-R
//                     decimation-in-frequency pre-step fused into the loads,
//                     so group r produces the outputs k = r (mod R).
//
// Sign convention: DIR = -1 is the forward transform X[k] = sum x[n] e^{-2 pi i kn/N},
// DIR = +1 the unnormalised inverse.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "df32.cuh"

namespace cmif {

template <typename T>
struct cpx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// FP32: one packed two-lane instruction per complex add / subtract (sm_100+
// FADD2 / FFMA2; each lane rounds like the scalar op, a - b as fma(b, -1, a)).
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return {r.x, r.y};
}
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) {
    const float2 r = __ffma2_rn(make_float2(b.x, b.y), make_float2(-1.f, -1.f), make_float2(a.x, a.y));
    return {r.x, r.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// multiply by e^{DIR * i * theta} given (cos theta, sin theta)
template <int DIR, typename T>
__device__ __forceinline__ cpx<T> rot(cpx<T> a, T c, T s) {
    if (DIR < 0) return {a.x * c + a.y * s, a.y * c - a.x * s};
    return {a.x * c - a.y * s, a.y * c + a.x * s};
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int brev(int k, int M) {
    int r = 0;
    for (int b = 1, t = M >> 1; b < M; b <<= 1, t >>= 1)
        if (k & b) r |= t;
    return r;
}

// cos / sin of 2*pi*k/32 from first-octant constants, so that the symmetric
// entries are exact mirror images.
__host__ __device__ constexpr double c16(int r) {
    return r == 0 ? 1.0 : r == 1 ? 0.98078528040323044913 : r == 2 ? 0.92387953251128675613
         : r == 3 ? 0.83146961230254523708 : 0.70710678118654752440;
}
__host__ __device__ constexpr double s16(int r) {
    return r == 0 ? 0.0 : r == 1 ? 0.19509032201612826785 : r == 2 ? 0.38268343236508977173
         : r == 3 ? 0.55557023301960222474 : 0.70710678118654752440;
}
__host__ __device__ constexpr double cos32q(int k) { return k <= 4 ? c16(k) : s16(8 - k); }   // k in [0, 8]
__host__ __device__ constexpr double sin32q(int k) { return k <= 4 ? s16(k) : c16(8 - k); }
__host__ __device__ constexpr double cos32(int k) {
    return k < 8 ? cos32q(k) : k < 16 ? -sin32q(k - 8) : k < 24 ? -cos32q(k - 16) : sin32q(k - 24);
}
__host__ __device__ constexpr double sin32(int k) {
    return k < 8 ? sin32q(k) : k < 16 ? cos32q(k - 8) : k < 24 ? -sin32q(k - 16) : -cos32q(k - 24);
}

// d * e^{DIR * 2 pi i k / M}, with the trivial angles special-cased.
template <int M, int DIR, typename T>
__device__ __forceinline__ cpx<T> twc(cpx<T> d, int k) {
    const int k32 = k * (32 / M);
    if (k32 == 0) return d;
    if (k32 == 8) return DIR < 0 ? cpx<T>{d.y, -d.x} : cpx<T>{-d.y, d.x};
    if (k32 == 16) return {-d.x, -d.y};
    if (k32 == 24) return DIR < 0 ? cpx<T>{-d.y, d.x} : cpx<T>{d.y, -d.x};
    return rot<DIR>(d, (T)cos32(k32), (T)sin32(k32));
}

// In-register M-point DFT, natural order in, bit-reversed order out:
// after the call v[brev(k, M)] = sum_n v_in[n] e^{DIR 2 pi i n k / M}.
// PACK = false keeps the butterflies' adds in scalar form (the +-i twiddles then
// stay free operand negations), for kernels where that issues fewer instructions.
template <int M, int DIR, bool PACK, typename T>
__device__ __forceinline__ void dft_reg_r22(cpx<T> (&v)[M]) {
    // Radix-2^2 ordering of the radix-2 network: the stages go in pairs; on the first
    // stage of a pair a lower output keeps only the quarter-turn part of its twiddle
    // (a free swap / negation) and defers the rest, which is the same for the two
    // inputs of its next butterfly and so moves past it; the second stage applies
    // everything pending.  N = 32: 28 general rotations instead of 34 (16: 8 vs 10).
    // pend[i]: rotation still owed by v[i], in units of 2 pi / 32 (all compile-time).
    int pend[M];
#pragma unroll
    for (int i = 0; i < M; ++i) pend[i] = 0;
#pragma unroll
    for (int span = M / 2, stage = 0; span >= 1; span >>= 1, ++stage) {
        const bool first = (stage % 2 == 0) && span >= 2;
#pragma unroll
        for (int start = 0; start < M; start += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const cpx<T> a = v[start + j], b = v[start + j + span];
                if constexpr (PACK) {
                    v[start + j] = a + b;
                    v[start + j + span] = a - b;
                } else {
                    v[start + j] = cpx<T>{a.x + b.x, a.y + b.y};
                    v[start + j + span] = cpx<T>{a.x - b.x, a.y - b.y};
                }
                pend[start + j + span] = (pend[start + j] + j * (32 / (2 * span))) & 31;
            }
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int e = pend[i];
            const int q = first ? (e & ~7) : e;
            if (q) v[i] = twc<32, DIR>(v[i], q);
            pend[i] = e - q;
        }
    }
}

template <int M, int DIR, bool PACK = true, bool R22 = false, typename T>
__device__ __forceinline__ void dft_reg(cpx<T> (&v)[M]) {
    if constexpr (R22) {
        dft_reg_r22<M, DIR, PACK>(v);
        return;
    }
#pragma unroll
    for (int span = M / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int start = 0; start < M; start += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; ++j) {
                cpx<T> a = v[start + j], b = v[start + j + span];
                if constexpr (PACK) {
                    v[start + j] = a + b;
                    v[start + j + span] = twc<M, DIR>(a - b, j * (M / (2 * span)));
                } else {
                    v[start + j] = cpx<T>{a.x + b.x, a.y + b.y};
                    v[start + j + span] = twc<M, DIR>(cpx<T>{a.x - b.x, a.y - b.y}, j * (M / (2 * span)));
                }
            }
        }
    }
}

}  // namespace cmif

namespace cmif {

// Lanes per group for a team transform: the largest power of two M with M*M
// dividing N (N = R M^2; for N = 2^k or 3 * 2^k), capped so that M complex
// values fit in registers (32 for FP32, 16 for FP64).
__host__ __device__ constexpr int team_m(int N, int mmax) {
    int M = mmax;
    while (M > 1 && (M * M > N || N % (M * M) != 0)) M >>= 1;
    return M;
}
__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// In-register R-point DFT with the output in natural order: u[q] = sum_s u_in[s]
// e^{DIR 2 pi i s q / R}.  Powers of two by the radix-2 network (the bit-reversed
// output renamed), R = 3 directly, R = 6 as two 3-point DFTs and a radix-2 step.
template <int DIR, typename T>
__device__ __forceinline__ void dft3(cpx<T>& a, cpx<T>& b, cpx<T>& c) {
    // X0 = a + b + c; X1,2 = a - (b + c)/2 -+ DIR i (sqrt(3)/2) (b - c) ... with the sign of DIR
    const T h = T(0.5), s3 = T(0.86602540378443864676);
    const cpx<T> t = {b.x + c.x, b.y + c.y}, d = {b.x - c.x, b.y - c.y};
    const cpx<T> m = {a.x - h * t.x, a.y - h * t.y};
    const cpx<T> id = {-s3 * d.y, s3 * d.x};  // i sqrt(3)/2 (b - c)
    a = {a.x + t.x, a.y + t.y};
    if (DIR > 0) {
        b = {m.x + id.x, m.y + id.y};
        c = {m.x - id.x, m.y - id.y};
    } else {
        b = {m.x - id.x, m.y - id.y};
        c = {m.x + id.x, m.y + id.y};
    }
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_nat(cpx<T> (&u)[R]) {
    if constexpr (R == 3) {
        dft3<DIR>(u[0], u[1], u[2]);
    } else if constexpr (R == 6) {
        // E = DFT3(u0, u2, u4), O = DFT3(u1, u3, u5); X[k] = E[k] + w6^k O[k], X[k+3] = E[k] - w6^k O[k]
        cpx<T> e0 = u[0], e1 = u[2], e2 = u[4], o0 = u[1], o1 = u[3], o2 = u[5];
        dft3<DIR>(e0, e1, e2);
        dft3<DIR>(o0, o1, o2);
        const T h = T(0.5), s3 = T(0.86602540378443864676);
        const cpx<T> w1 = {h, DIR * s3}, w2 = {-h, DIR * s3};
        o1 = cmul(o1, w1);
        o2 = cmul(o2, w2);
        u[0] = e0 + o0; u[3] = e0 - o0;
        u[1] = e1 + o1; u[4] = e1 - o1;
        u[2] = e2 + o2; u[5] = e2 - o2;
    } else {
        static_assert(is_pow2(R), "R-point DFT: powers of two, 3 and 6");
        cpx<T> t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = u[i];
        dft_reg<R, DIR>(t);
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = t[brev(q, R)];
    }
}
template <typename T>
__host__ __device__ constexpr int max_m() { return sizeof(T) == 4 ? 32 : 16; }  // FP32: 32; FP64 and two-term FP32: 16

// Twiddle tables in device memory, filled once per device from FP64 values.
//   n[l][k]         = e^{-2 pi i k / 2^l},           k < 2^l
//   sq[l][k1*M + j] = e^{-2 pi i j k1 / (M*M)},       M = 2^l, j, k1 < M
//   n3[l][k]        = e^{-2 pi i k / (3 2^l)},       k < 3 2^l
template <typename T>
struct Tw {
    const cpx<T>* n[14];
    const cpx<T>* sq[6];
    const cpx<T>* n3[12];
};

// The table of e^{-2 pi i k / N} for a transform length N = 2^l or 3 2^l.
__host__ __device__ constexpr int ilog2_of(int n) { return n <= 1 ? 0 : 1 + ilog2_of(n >> 1); }
template <int N, typename T>
__device__ __forceinline__ const cpx<T>* tw_of(const Tw<T>& tw) {
    if constexpr (N % 3 == 0) return tw.n3[ilog2_of(N / 3)];
    else return tw.n[ilog2_of(N)];
}

template <int DIR, typename T>
__device__ __forceinline__ cpx<T> twl(const cpx<T>* __restrict__ t, int k) {
    cpx<T> w = t[k];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// Shared-memory scratch of one group of M lanes.  FP32 transposes go through
// shared memory in two halves (real parts, then imaginary parts), so a group
// needs M*M floats; groups narrower than a warp get M floats of padding so
// that the groups of one warp hit disjoint banks.  FP64 transposes complex
// values directly.
template <int M>
__host__ __device__ constexpr int grp_pad() { return M < 32 ? M : 0; }
template <typename T, int M>
__host__ __device__ constexpr int grp_scratch_bytes() {
    return sizeof(T) == 4 ? (M * M + grp_pad<M>()) * 4 : M * M * (int)sizeof(cpx<T>);
}

// Shared memory of one team of R groups: the groups' scratch, or for R > 2 the
// N complex values of the radix-R exchange if that is more.
template <typename T, int M, int R>
__host__ __device__ constexpr int team_scratch_bytes() {
    return R > 2 && R * M * M * (int)sizeof(cpx<T>) > R * grp_scratch_bytes<T, M>()
               ? R * M * M * (int)sizeof(cpx<T>) : R * grp_scratch_bytes<T, M>();
}

// Length N = R*M*M transform by a team of R groups x M lanes.
//   load(n)  : x[n] for n in [0, N)
//   r, j     : this lane's group and lane-in-group
//   sm       : this group's scratch (grp_scratch_bytes<T, M>() bytes of shared memory);
//              for R > 2 the team's groups' scratch must start at sm - r * grp_scratch and
//              span at least N complex values (team_scratch_bytes)
//   twq      : Tw::sq for this M;  twn : Tw::n for N (used when R > 1)
// Result: v[brev(k2, M)] = X[R*(j + M*k2) + r], k2 in [0, M).
// Every lane of every warp taking part must call this (it uses __syncwarp).
// The four-step core on values already in registers: v[i] = y[j + M*i] for the
// group's M*M-point sequence y.  Result: v[brev(k2, M)] = Y[j + M*k2].
// R22: bit 0 / bit 1 put the first / second register DFT in the radix-2^2 order.
template <int M, int DIR, bool PACK = true, bool WIDE = false, int R22 = 0, typename T>
__device__ __forceinline__ void team_fft_core(cpx<T> (&v)[M], int j, void* sm, const cpx<T>* __restrict__ twq) {
    dft_reg<M, DIR, PACK, (R22 & 1) != 0>(v);  // v[brev(k1)] = A[j][k1]
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) v[brev(k1, M)] = cmul(v[brev(k1, M)], twl<DIR>(twq, k1 * M + j));
    if constexpr (WIDE) {
        // WIDE (FP32, M = 16 or 32, a group scratch of M*M complex): one pass of complex
        // values.  Row k1 holds M/2 blocks of two complex; element (k1, col) sits in
        // block (col / 2) ^ (k1 % 8).  A row write by the 32 lanes is a permutation of
        // the row; the 16-byte row reads of 8 lanes (rows j .. j + 7) hit 8 different
        // 16-byte bank groups: conflict-free.
        static_assert(sizeof(T) == 4 && (M == 32 || M == 16), "wide transpose: FP32, 16- or 32-lane groups");
        float2* sc = reinterpret_cast<float2*>(sm);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            const cpx<T> z = v[brev(k1, M)];
            sc[k1 * M + ((((j >> 1) ^ (k1 & 7)) << 1) | (j & 1))] = make_float2(z.x, z.y);
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < M / 2; ++b) {
            const float4 q = *reinterpret_cast<const float4*>(sc + j * M + ((b ^ (j & 7)) << 1));
            v[2 * b] = {q.x, q.y};
            v[2 * b + 1] = {q.z, q.w};
        }
        __syncwarp();
    } else if constexpr (sizeof(T) == 4 && M == 32) {
        // Rows of 32 floats in 8 blocks of 4; element (row, col) sits in block
        // (col/4) ^ (row % 8).  Column writes (one float per lane) are a
        // permutation of the row's 32 banks; row reads take 16-byte loads and the
        // 8 lanes of each 16-byte phase hit 8 different blocks: conflict-free.
        float* sf = reinterpret_cast<float*>(sm);
        const int jb = j >> 2, jl = j & 3;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            __syncwarp();
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1)
                sf[k1 * M + (((jb ^ k1) & 7) << 2) + jl] = half ? v[brev(k1, M)].y : v[brev(k1, M)].x;
            __syncwarp();
#pragma unroll
            for (int b4 = 0; b4 < 8; ++b4) {
                const float4 q = *reinterpret_cast<const float4*>(sf + j * M + (((b4 ^ j) & 7) << 2));
                if (half) { v[4 * b4].y = q.x; v[4 * b4 + 1].y = q.y; v[4 * b4 + 2].y = q.z; v[4 * b4 + 3].y = q.w; }
                else      { v[4 * b4].x = q.x; v[4 * b4 + 1].x = q.y; v[4 * b4 + 2].x = q.z; v[4 * b4 + 3].x = q.w; }
            }
        }
        __syncwarp();
    } else if constexpr (sizeof(T) == 4) {
        float* sf = reinterpret_cast<float*>(sm);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) sf[k1 * M + (j ^ k1)] = v[brev(k1, M)].x;
        __syncwarp();
#pragma unroll
        for (int n2 = 0; n2 < M; ++n2) v[n2].x = sf[j * M + (n2 ^ j)];
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) sf[k1 * M + (j ^ k1)] = v[brev(k1, M)].y;
        __syncwarp();
#pragma unroll
        for (int n2 = 0; n2 < M; ++n2) v[n2].y = sf[j * M + (n2 ^ j)];
        __syncwarp();
    } else {
        cpx<T>* sc = reinterpret_cast<cpx<T>*>(sm);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) sc[k1 * M + (j ^ k1)] = v[brev(k1, M)];
        __syncwarp();
#pragma unroll
        for (int n2 = 0; n2 < M; ++n2) v[n2] = sc[j * M + (n2 ^ j)];
        __syncwarp();
    }
    dft_reg<M, DIR, PACK, (R22 & 2) != 0>(v);  // v[brev(k2)] = X_r[j + M k2]
}

template <int M, int R, int DIR, bool PACK = true, bool ONCE = false, bool WIDE = false, int R22 = 0,
          typename T, typename Load>
__device__ __forceinline__ void team_fft(cpx<T> (&v)[M], int r, int j, Load&& load, void* sm,
                                         const cpx<T>* __restrict__ twq, const cpx<T>* __restrict__ twn) {
    // WIDE: the groups' scratch are M*M complex each (one-pass complex transposes);
    // sm is then this group's slice at r * M*M complex from the team's base
    // ONCE (R = 2, teams of one warp): the radix-2 step loads every input once and
    // passes the groups' halves through the team's buffer (2 M^2 complex values in
    // front of the groups' scratch), instead of each group loading all inputs.
    constexpr int NQ = M * M;
    if constexpr (ONCE) {
        static_assert(R == 2 && R * M == 32, "load-once radix-2 step: one-warp teams");
        constexpr int H2 = M / 2;
        constexpr int GS = WIDE ? M * M * (int)sizeof(cpx<T>) : grp_scratch_bytes<T, M>();
        cpx<T>* xs = reinterpret_cast<cpx<T>*>(reinterpret_cast<char*>(sm) - r * GS);
        __syncwarp();  // earlier users of the team's scratch are done
#pragma unroll
        for (int t = 0; t < H2; ++t) {
            const int m = j + M * (r * H2 + t);  // the lanes of both groups cover m < NQ once
            const cpx<T> x0 = load(m), x1 = load(m + NQ);
            xs[m] = x0 + x1;
            xs[NQ + m] = cmul(x0 - x1, twl<DIR>(twn, m));
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = xs[r * NQ + j + M * i];
        __syncwarp();  // the groups' transposes below reuse this buffer
    } else if constexpr (R > 2 && !is_pow2(R)) {
        // Radix-R decimation in frequency (R = 3, 6) with every input loaded once: the
        // team's lanes l = r M + j take the points m = l + TEAM t, form the R-point DFT
        // of x[m + s NQ], s < R, twiddle frequency q by w_N^{m q} and hand it to group q
        // through the team's buffer (as in the power-of-two case below).
        constexpr int TEAM = R * M, PTS = (NQ + TEAM - 1) / TEAM;
        cpx<T>* xs = reinterpret_cast<cpx<T>*>(reinterpret_cast<char*>(sm) - r * grp_scratch_bytes<T, M>());
        const int lt = r * M + j;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < PTS; ++t) {
            const int m = lt + TEAM * t;
            if (PTS * TEAM == NQ || m < NQ) {
                cpx<T> u[R];
#pragma unroll
                for (int s2 = 0; s2 < R; ++s2) u[s2] = load(m + s2 * NQ);
                dft_nat<R, DIR>(u);
#pragma unroll
                for (int q = 0; q < R; ++q) xs[q * NQ + m] = q ? cmul(u[q], twl<DIR>(twn, m * q)) : u[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = xs[r * NQ + j + M * i];
        __syncthreads();
    } else if constexpr (R > 2) {
        // Radix-R decimation in frequency with every input loaded once: lane (r, j)
        // takes the points m = j + M (r PER + t), t < PER, forms the R-point DFT of
        // x[m + s NQ], s < R, in registers, twiddles frequency q by w_N^{m q} and
        // hands it to group q through the team's buffer (N complex values in front
        // of the groups' scratch: sm - r * grp_scratch).  Block-wide barriers: every
        // team of the block must call this together.
        constexpr int PER = M / R;
        static_assert(PER >= 1, "radix-R step needs R <= M");
        cpx<T>* xs = reinterpret_cast<cpx<T>*>(reinterpret_cast<char*>(sm) - r * grp_scratch_bytes<T, M>());
        __syncthreads();  // earlier users of the team's scratch are done
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int m = j + M * (r * PER + t);
            cpx<T> u[R];
#pragma unroll
            for (int s2 = 0; s2 < R; ++s2) u[s2] = load(m + s2 * NQ);
            dft_reg<R, DIR, PACK>(u);  // u[brev(q)] = sum_s x[m + s NQ] w_R^{s q}
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const cpx<T> y = u[brev(q, R)];
                xs[q * NQ + m] = q ? cmul(y, twl<DIR>(twn, m * q)) : y;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = xs[r * NQ + j + M * i];
        __syncthreads();  // the groups' transposes below reuse this buffer
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int m = j + M * i;
            if constexpr (R == 1) {
                v[i] = load(m);
            } else {
                // radix-2 decimation in frequency: y_r[m] = w_N^{m r} (x[m] + (-1)^r x[m + NQ])
                const cpx<T> x0 = load(m), x1 = load(m + NQ);
                const cpx<T> acc = (r & 1) ? x0 - x1 : x0 + x1;
                v[i] = (r == 0) ? acc : cmul(acc, twl<DIR>(twn, m * r));
            }
        }
    }
    team_fft_core<M, DIR, PACK, WIDE, R22>(v, j, sm, twq);
}

}  // namespace cmif
