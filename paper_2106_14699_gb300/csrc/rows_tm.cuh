// Inverse row transform + fused entropy epilogue, FP32, one warp per pair
// transform (Q = 512, 1024 or 2048), with
//   * the B-marginal accumulators C_B^b(p) held in Tensor Memory (TMEM,
//     tcgen05.ld / tcgen05.st), one 32-bit column per (b, position) of the
//     owning thread, and
//   * each team's next Y row fetched into shared memory by a TMA bulk copy
//     (cp.async.bulk + mbarrier) while the current round computes.
// Same arithmetic and outputs as k_pair_rows (kernels.cuh), except the debug
// count maps: a call that asks for them runs k_pair_rows.
#pragma once
#include "kernels.cuh"

namespace cmif {

// ---- mbarrier / TMA bulk copy ------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(phase) : "memory");
    return done != 0;
}
// Bounded wait: gives up after `polls` polls (by default 2^24, far beyond any
// copy's latency) and returns false, so that a lost copy can never hang the GPU.
constexpr int kDefaultWaitPolls = 1 << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, int polls = kDefaultWaitPolls) {
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// ---- Tensor Memory ------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[N]);
template <int N>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t (&r)[N]);

template <>
__device__ __forceinline__ void tmem_ld<1>(uint32_t t, uint32_t (&r)[1]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[0]) : "r"(t) : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<1>(uint32_t t, const uint32_t (&r)[1]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(t), "r"(r[0]) : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<2>(uint32_t t, uint32_t (&r)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(t) : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<2>(uint32_t t, const uint32_t (&r)[2]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(t), "r"(r[0]), "r"(r[1]) : "memory");
}
#define CMIF_R16(o) "=r"(r[o]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), "=r"(r[o + 5]), \
    "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), "=r"(r[o + 11]),           \
    "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
#define CMIF_W16(o) "r"(r[o]), "r"(r[o + 1]), "r"(r[o + 2]), "r"(r[o + 3]), "r"(r[o + 4]), "r"(r[o + 5]), \
    "r"(r[o + 6]), "r"(r[o + 7]), "r"(r[o + 8]), "r"(r[o + 9]), "r"(r[o + 10]), "r"(r[o + 11]),           \
    "r"(r[o + 12]), "r"(r[o + 13]), "r"(r[o + 14]), "r"(r[o + 15])
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t t, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15}, [%16];"
                 : CMIF_R16(0) : "r"(t) : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<16>(uint32_t t, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};"
                 ::"r"(t), CMIF_W16(0) : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t t, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : CMIF_R16(0), CMIF_R16(16) : "r"(t) : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<32>(uint32_t t, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 ::"r"(t), CMIF_W16(0), CMIF_W16(16) : "memory");
}
#undef CMIF_R16
#undef CMIF_W16

// ---------------------------------------------------------------------------
template <int Q>
struct RowTmCfg {
    static constexpr int L = Q / 2;
    // Q = 512: a one-warp team needs M = 8, R = 4 (256 = 4 * 8^2).  Q <= 1024: one
    // pass holds the whole row (the team's scratch has room for it: at 1024 the
    // load-once radix-2 buffer), fewer barriers and TMEM round trips per round
    static constexpr int MMAX = Q <= 512 ? 8 : 32;
    static constexpr int HALVES = Q <= 1024 ? 1 : 2;
    using G = TeamGeom<float, L, MMAX>;
    static constexpr int M = G::M, R = G::R, TEAM = G::TEAM;
    static constexpr int NT = 16, THREADS = NT * 32;
    static constexpr int QH = Q / HALVES;        // positions per pass
    static constexpr int UH = QH / THREADS;      // positions per thread per pass: UH t .. UH t + UH - 1 (adjacent,
                                                 // so that the counts of one thread come in one shared load)
    static constexpr int U = HALVES * UH;
    // radix-2 teams (Q = 1024) load every input once through a buffer of 2 M^2 complex
    static constexpr bool ONCE = R == 2;
    static constexpr int XS = ONCE ? R * M * M * 8 : 0;
    static constexpr int REGION = G::SCRATCH > XS ? G::SCRATCH : XS;  // FFT scratch / one pass of rounded counts
    static constexpr int STAGE_BYTES = ((L + 1) * 8 + 15) / 16 * 16;  // one Y row (Qh complex), 16-byte multiple
    static constexpr size_t OFF_STAGE = (size_t)NT * REGION;
    static constexpr size_t OFF_BAR = OFF_STAGE + (size_t)NT * STAGE_BYTES;
    static constexpr size_t OFF_HOLD = OFF_BAR + NT * 8;
    static constexpr int NQ = M * M;
    static constexpr int TW_PRE = R > 1 ? (R - 1) * NQ + 1 : 0;
    static constexpr size_t OFF_TW = OFF_HOLD + 16;                   // twiddles staged in shared memory:
    static constexpr size_t SMEM = OFF_TW + (size_t)(NQ + L + TW_PRE) * 8;  // four-step, C2R, pre-step
    static_assert(TEAM == 32, "one warp per transform");
    static_assert(UH >= 1 && QH % THREADS == 0, "whole positions per thread");
    static_assert(REGION >= QH * 4, "scratch holds one pass");
};

// TMEM columns one thread needs: K_B marginals x U positions; four warps share a lane quadrant.
__host__ __device__ constexpr int tm_cols_needed(int KB, int U) { return 4 * KB * U; }
__host__ __device__ constexpr int tm_alloc_cols(int need) {
    return need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}

// MODE 0 is the plain FP32 kernel (one map); MODE 1 takes several units per
// launch (rotation angles); MODE 2 adds to that the per-pair precision of
// CMIF_AUTO (conditional re-run, exact counts of listed pairs, per-pair
// residuals) and the diagnostics of the bounded waits (poll limit, withheld
// copy).  They are separate instantiations because the plain kernel sits at
// the register limit.
template <int Q, bool NMI, int MODE>
__global__ void __launch_bounds__(RowTmCfg<Q>::THREADS, 1)
k_pair_rows_tm(const cpx<float>* __restrict__ Y, Geom g, Tw<float> tw, double* __restrict__ mi_map,
               int32_t* __restrict__ n_map, DevStatus* __restrict__ st,
               int tm_cols, int wait_polls, int withhold_row, int conditional, const int32_t* __restrict__ ov,
               const int* __restrict__ ov_slot, unsigned* __restrict__ pair_res) {
    // wait_polls: poll limit of the bounded waits.  withhold_row >= 0 (diagnostics
    // only): the bulk copy of that output row's first pair is never issued, so the
    // wait for it runs out and the kernel takes its timeout path.  conditional: run
    // only when the status word asks for the re-run.  ov, ov_slot, pair_res: the
    // exact counts of second-precision pairs and the per-pair residuals, as in
    // k_pair_rows.
    using C = RowTmCfg<Q>;
    constexpr bool EXT = MODE == 2, MULTI = MODE >= 1;
    if (EXT && conditional && !(st->flags & STATUS_ESCALATE)) return;  // uniform, before any set-up
    if (!EXT) {
        wait_polls = kDefaultWaitPolls;
        withhold_row = -1;
    }
    constexpr int M = C::M, R = C::R, L = C::L, NT = C::NT, U = C::U, UH = C::UH, QH = C::QH, HALVES = C::HALVES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, team = tid >> 5, lane = tid & 31, r = lane / M, j = lane % M;
    unsigned char* region = smem_raw + (size_t)team * C::REGION;
    const cpx<float>* stage = reinterpret_cast<const cpx<float>*>(smem_raw + C::OFF_STAGE + (size_t)team * C::STAGE_BYTES);
    const uint32_t stage_s = smem_u32(stage);
    const uint32_t bar = smem_u32(smem_raw + C::OFF_BAR + team * 8);
    uint32_t* hold = reinterpret_cast<uint32_t*>(smem_raw + C::OFF_HOLD);
    __shared__ int s_abort;

    const int KA = g.KA, KB = g.KB, npairs = KA * KB, Rout = g.R, Cout = g.C, Qs = g.Qs;
    cpx<float>* tw_sq = reinterpret_cast<cpx<float>*>(smem_raw + C::OFF_TW);
    cpx<float>* twq_c2r = tw_sq + C::NQ;
    cpx<float>* tw_pre = twq_c2r + L;
    stage_table(tw_sq, tw.sq[ilog2c(M)], C::NQ);
    stage_table(twq_c2r, tw_of<Q>(tw), L);
    if (R > 1) stage_table(tw_pre, tw_of<L>(tw), C::TW_PRE);

    if (tid == 0) s_abort = 0;
    if (lane == 0) mbar_init(bar, 1);
    if (team == 0) tmem_alloc(smem_u32(hold), (uint32_t)tm_cols);
    mbar_fence_init();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *hold;
    // this warp's TMEM slice: lanes of quadrant (warp % 4), columns of block (warp / 4)
    const uint32_t tbase = tmem + ((uint32_t)(32 * (team & 3)) << 16) + (uint32_t)((team >> 2) * KB * U);

    // work items of this team: (row, base) in order; prefetch the first active one
    uint32_t phase = 0;
    bool pending = false;  // a copy issued for this team and not yet waited for
    // work: the window's rows r0 + blockIdx.x + k * gridDim.x of every unit (units > 1:
    // several maps, R2 rows apart), unit by unit
    auto issue = [&](int row_i, int pair_i) {
        if (EXT && row_i == withhold_row && pair_i == 0) return;  // diagnostics: leave this wait without its copy
        if (lane == 0) {
            fence_proxy_async_smem();
            const cpx<float>* src = Y + ((size_t)pair_i * Rout + row_i) * Qs;
            tma_bulk_g2s(stage_s, src, C::STAGE_BYTES, bar);
        }
        pending = true;
    };
    if (g.r0 + (int)blockIdx.x < g.r1 && team < npairs) issue(g.r0 + blockIdx.x, team);

    float res_max = 0.f;
    int row_max_n = 0;
    bool aborted = false;
    int rbase = 0;  // first map row of the current unit (multi-unit kernels: unit * R2, up to R)
    for (int rr = g.r0 + blockIdx.x; rr < g.r1 && !aborted; rr += gridDim.x) {
        const int row = MULTI ? rbase + rr : rr;
        EntAcc<NMI> S[U];
        float CA[U];
        int N[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { S[u].zero(); CA[u] = 0.f; N[u] = 0; }
        {   // zero this thread's B-marginal columns
            uint32_t z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = 0u;
            for (int c0 = 0; c0 < KB * U; c0 += 16) {
                if (c0 + 16 <= KB * U) tmem_st<16>(tbase + c0, z);
                else for (int c = c0; c < KB * U; ++c) { uint32_t z1[1] = {0u}; tmem_st<1>(tbase + c, z1); }
            }
            tmem_wait_st();
        }
        int cur_a[2] = {0, 0};
        for (int base = 0; base < npairs; base += NT) {
            const int pair = base + team;
            const bool act = pair < npairs;
            if (act) {
                if (mbar_wait_bounded(bar, phase, wait_polls)) {
                    phase ^= 1u;
                    pending = false;
                } else {
                    atomicOr(&st->flags, STATUS_TIMEOUT);
                    s_abort = 1;
                }
            }
            // Hermitian split: z = IDFT_L(E + iO), z[m] = x[2m] + i x[2m+1].  With
            // t = e^{-2 pi i k/Q} from the table: E = y_k + conj(y_{L-k}),
            // iO = (y_k - conj(y_{L-k})) * i conj(t) = d * (t.y, t.x); packed adds.
            auto load = [&](int k) -> cpx<float> {
                if (!act) return {0.f, 0.f};
                const float2 yk = reinterpret_cast<const float2*>(stage)[k];
                const float2 ym = reinterpret_cast<const float2*>(stage)[L - k];
                const float2 e = __ffma2_rn(ym, make_float2(1.f, -1.f), yk);
                const float2 d = __ffma2_rn(ym, make_float2(-1.f, 1.f), yk);
                const cpx<float> t = twq_c2r[k];
                const cpx<float> io = cmul(cpx<float>{d.x, d.y}, cpx<float>{t.y, t.x});
                const float2 z = __fadd2_rn(e, make_float2(io.x, io.y));
                return {z.x, z.y};
            };
            cpx<float> v[M];
            if constexpr (R == 1 && M == 32 && C::STAGE_BYTES >= M * M * 8) {
                // the staged row is consumed by the loads: its buffer takes the one-pass
                // complex transpose (the next copy into it is issued after the transform)
#pragma unroll
                for (int i = 0; i < M; ++i) v[i] = load(j + M * i);
                team_fft_core<M, +1, false, true, 3>(v, j, const_cast<cpx<float>*>(stage), tw_sq);
            } else {
                team_fft<M, R, +1, false, C::ONCE, false, 3>(v, r, j, load, region + r * grp_scratch_bytes<float, M>(),
                                                                 tw_sq, tw_pre);
            }
            // the staging buffer is free again: prefetch this team's next active item
            // (the next round of this row, else round 0 of its next row)
            __syncwarp();
            if (act && !pending) {
                if constexpr (MULTI) {
                    int nb = rbase, nrr = rr, npair = pair + NT;
                    if (npair >= npairs) {
                        npair = team;
                        nrr = rr + gridDim.x;
                        if (nrr >= g.r1) { nrr = g.r0 + blockIdx.x; nb += g.R2; }
                    }
                    if (nb < g.R && nrr < g.r1) issue(nb + nrr, npair);
                } else {
                    int nrow = row, npair = pair + NT;
                    if (npair >= npairs) { nrow = row + gridDim.x; npair = team; }
                    if (nrow < g.r1) issue(nrow, npair);
                }
            }
            float rp = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                // nearest integers (the 1.5 * 2^23 shift, packed) and the residual
                const float2 x = make_float2(v[k].x, v[k].y);
                const float2 c = __fadd2_rn(__fadd2_rn(x, make_float2(12582912.0f, 12582912.0f)),
                                            make_float2(-12582912.0f, -12582912.0f));
                const float2 dv = __ffma2_rn(c, make_float2(-1.f, -1.f), x);
                if constexpr (EXT) rp = fmaxf(rp, fmaxf(fabsf(dv.x), fabsf(dv.y)));
                else res_max = fmaxf(res_max, fmaxf(fabsf(dv.x), fabsf(dv.y)));
                v[k].x = c.x;
                v[k].y = c.y;
            }
            const int ovs = (EXT && act && ov_slot) ? ov_slot[pair] : -1;  // loaded after the transform: fewer live registers
            if (EXT && ovs < 0) res_max = fmaxf(res_max, rp);
            if (EXT && pair_res && act && ovs < 0) {  // the warp is this pair's team
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) rp = fmaxf(rp, __shfl_xor_sync(0xffffffffu, rp, off));
                if (lane == 0) atomic_max_float_pos(&pair_res[pair], rp);
            }
            const int nt = min(NT, npairs - base);
            const int a0 = base / KB, b0 = base - a0 * KB;
            const bool fast = (KB == NT) && (b0 == 0);  // the round is exactly (a0, b = 0..15)
#pragma unroll
            for (int hf = 0; hf < HALVES; ++hf) {
                __syncthreads();
                float2* ob = reinterpret_cast<float2*>(region);
                if (EXT && ovs >= 0) {  // exact counts of positions 2 mf, 2 mf + 1 from the second precision
                    const int32_t* ovr = ov + ((size_t)ovs * Rout + row) * Q;
#pragma unroll
                    for (int k2 = hf * (M / HALVES); k2 < (hf + 1) * (M / HALVES); ++k2) {
                        const int mf = R * (j + M * k2) + r;
                        const int2 q = *reinterpret_cast<const int2*>(ovr + 2 * mf);
                        ob[mf - hf * (L / HALVES)] = make_float2((float)q.x, (float)q.y);
                    }
                } else {
#pragma unroll
                    for (int k2 = hf * (M / HALVES); k2 < (hf + 1) * (M / HALVES); ++k2) {
                        const int m = R * (j + M * k2) + r - hf * (L / HALVES);
                        const cpx<float> z = v[brev(k2, M)];
                        ob[m] = make_float2(z.x, z.y);
                    }
                }
                __syncthreads();
                const uint32_t tcol = tbase + (uint32_t)(hf * KB * UH);
                if (fast) {
                    // all 16 B-marginals of this pass in registers: one TMEM load / store
                    if (a0 != cur_a[hf]) {
#pragma unroll
                        for (int uh = 0; uh < UH; ++uh) {
                            const int u = hf * UH + uh;
                            S[u].marg(clog2c_fixed(CA[u]));
                            N[u] += (int)CA[u];
                            CA[u] = 0.f;
                        }
                        cur_a[hf] = a0;
                    }
                    uint32_t cbr[16 * UH];
                    if constexpr (UH == 2) tmem_ld<32>(tcol, cbr);
                    else tmem_ld<16>(tcol, cbr);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const float* obt = reinterpret_cast<const float*>(smem_raw + (size_t)t * C::REGION);
#pragma unroll
                        for (int uh = 0; uh < UH; ++uh) {
                            const int u = hf * UH + uh, pl = UH * tid + uh;
                            const float c = obt[pl];
                            S[u].joint(clog2c_fixed(c));
                            CA[u] += c;
                            cbr[t * UH + uh] = __float_as_uint(__uint_as_float(cbr[t * UH + uh]) + c);
                        }
                    }
                    if constexpr (UH == 2) tmem_st<32>(tcol, cbr);
                    else tmem_st<16>(tcol, cbr);
                    tmem_wait_st();
                } else {
                    int a = a0, b = b0;
                    for (int t = 0; t < nt; ++t) {
                        if (a != cur_a[hf]) {
#pragma unroll
                            for (int uh = 0; uh < UH; ++uh) {
                                const int u = hf * UH + uh;
                                S[u].marg(clog2c_fixed(CA[u]));
                                N[u] += (int)CA[u];
                                CA[u] = 0.f;
                            }
                            cur_a[hf] = a;
                        }
                        uint32_t cbr[UH];
                        tmem_ld<UH>(tcol + (uint32_t)(b * UH), cbr);
                        tmem_wait_ld();
                        const float* obt = reinterpret_cast<const float*>(smem_raw + (size_t)t * C::REGION);
#pragma unroll
                        for (int uh = 0; uh < UH; ++uh) {
                            const int u = hf * UH + uh, pl = UH * tid + uh;
                            const float c = obt[pl];
                            S[u].joint(clog2c_fixed(c));
                            CA[u] += c;
                            cbr[uh] = __float_as_uint(__uint_as_float(cbr[uh]) + c);
                        }
                        tmem_st<UH>(tcol + (uint32_t)(b * UH), cbr);
                        tmem_wait_st();
                        if (++b == KB) { b = 0; ++a; }
                    }
                }
            }
            __syncthreads();  // the next round's transforms overwrite the scratch read above
            if (s_abort) { aborted = true; break; }
        }
        if (aborted) break;
        // finish the row: last A-marginal, the B-marginals, MI
#pragma unroll
        for (int hf = 0; hf < HALVES; ++hf) {
#pragma unroll
            for (int uh = 0; uh < UH; ++uh) {
                const int u = hf * UH + uh;
                S[u].marg(clog2c_fixed(CA[u]));
                N[u] += (int)CA[u];
            }
            for (int b = 0; b < KB; ++b) {
                uint32_t cbr[UH];
                tmem_ld<UH>(tbase + (uint32_t)(hf * KB * UH + b * UH), cbr);
                tmem_wait_ld();
#pragma unroll
                for (int uh = 0; uh < UH; ++uh) {
                    const float cbv = __uint_as_float(cbr[uh]);
                    S[hf * UH + uh].marg(clog2c_fixed(cbv));
                }
            }
#pragma unroll
            for (int uh = 0; uh < UH; ++uh) {
                const int u = hf * UH + uh;
                const int cidx = circ_to_out(hf * QH + UH * tid + uh, Q, g.WA, g.WB - 1);
                if (cidx < 0) continue;
                const size_t o = (size_t)row * Cout + cidx;
                mi_map[o] = S[u].finish(N[u]);
                if (n_map) n_map[o] = N[u];
                if (cidx >= g.c0 && cidx < g.c1) row_max_n = max(row_max_n, N[u]);
            }
        }
        __syncthreads();
        if constexpr (MULTI) {  // past the unit's last row: the next unit's first
            if (rr + (int)gridDim.x >= g.r1 && rbase + g.R2 < g.R) {
                rbase += g.R2;
                rr = g.r0 + (int)blockIdx.x - (int)gridDim.x;
            }
        }
    }
    // A team may still have a copy in flight (prefetched for an item it will not run
    // after an abort): wait for it, bounded, before the block exits.
    if (pending) mbar_wait_bounded(bar, phase, wait_polls);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        res_max = fmaxf(res_max, __shfl_xor_sync(0xffffffffu, res_max, off));
        row_max_n = max(row_max_n, __shfl_xor_sync(0xffffffffu, row_max_n, off));
    }
    if (lane == 0) {
        atomic_max_float_pos(&st->res_bits[0], res_max);
        atomicMax(&st->max_n, row_max_n);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (team == 0) tmem_dealloc(tmem, (uint32_t)tm_cols);
}

}  // namespace cmif
