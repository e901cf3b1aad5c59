// C ABI of the CMIF library: plans, workspace, launch order, status.
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cmif.h"
#include "kernels.cuh"
#include "misc.h"
#include "pipeline.cuh"
#include "profiler.h"

using namespace cmif;

namespace {

template <typename T>
struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    PipeArgs<T> args{};  // pointer part filled at create time
    int rows_grid = 0;
    bool cb_smem = true;
    int rows_grid_w = 0;  // > 0: the plan computes weighted maps (FP64 workspace only)
    int ypairs = 0;       // pairs the Y buffer holds (0: all K_A * K_B; the second precision of AUTO: one chunk)
    // row-kernel alternatives (FP32): the Tensor-Memory kernel and the generic one
    int tm_cols_avail = 0;  // > 0: the TMEM kernel applies (its TMEM columns)
    int grid_tm = 0;        // its persistent grid
    int grid_gen = 0;       // the generic kernel's grid, when its B-marginals fit in shared memory (else 0)
};

// Per-pair precision of CMIF_AUTO: device buffers of the pair list and the exact
// counts of the listed pairs.
struct Escal {
    int* popA = nullptr;              // [K_A] label pixel counts (A)
    int* popB = nullptr;              // [K_B]
    unsigned char* needA = nullptr;   // [K_A] planes the second precision transforms
    unsigned char* needB = nullptr;   // [K_B]
    int* plist = nullptr;             // [K_A K_B] listed pairs, in slot order
    int* hdr = nullptr;               // [4] list ranges: stage 1 [hdr0, hdr1), stage 2 [hdr1, hdr2)
    int* ov_slot = nullptr;           // [K_A K_B] slot of a pair, -1 when not listed
    unsigned* pair_res = nullptr;     // [K_A K_B] FP32 residual per pair (float bits)
    int32_t* ov = nullptr;            // [cap][R][Q] exact counts of the listed pairs
    int cap = 0;                      // list capacity (slots)
    int chunk = 0;                    // pairs per second-precision chunk (its Y buffer)
    size_t bytes = 0;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr int kMaxAngles = 4096;

int pow2_at_least(int v, int lo) {
    int p = lo;
    while (p < v) p <<= 1;
    return p;
}

// Transform length for n outputs: the smallest power of two >= max(n, 16), or,
// for FP32 transforms, the smallest 3 * 2^k (96 .. 3072) if that is smaller.
int transform_size(int n, bool mixed) {
    int best = pow2_at_least(n, 16);
    if (mixed)
        for (int t = 96; t <= 3072; t <<= 1)
            if (t >= n && t < best) best = t;
    return best;
}

}  // namespace

struct cmif_plan_s {
    int device = 0;
    int num_sms = 0;
    Geom g{};
    cmif_precision prec = CMIF_FP32;
    unsigned flags = 0;
    Workspace<float> w32;
    Workspace<double> w64;
    Workspace<df32> ws32;  // two-term FP32 (split precision)
    bool has32 = false, has64 = false;
    cmif_precision tier2 = CMIF_SPLIT32;  // precision of AUTO's re-run
    DevStatus* st = nullptr;      // status of the map being computed (reset per map)
    DevStatus* st_total = nullptr;  // status of the whole call (what cmif_get_status reports)
    PeakPart* parts = nullptr;
    int nparts = 0;
    void* mem = nullptr;      // the plan's one device allocation (nullptr when a batch owns the memory)
    size_t mem_bytes = 0;
    size_t small_bytes = 0;
    int32_t* nbuf = nullptr;  // N map used when the caller passes no n_map
    double* mibuf = nullptr;  // MI map used by cmif_align_rotations when the caller keeps no maps
    int32_t* wB = nullptr;    // rotated floating image (cmif_align_rotations)
    uint8_t* wM = nullptr;    // its rotated-support mask
    void* peaks = nullptr;    // per-transform peaks, kMaxAngles records (+ 2 for the two-stage search)
    // host-buffer path staging (allocated lazily by cmif_compute_host)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t last_stream = nullptr;
    Profiler prof;
    // CUDA-graph replay (CMIF_FLAG_GRAPH): the captured launch sequence of the last
    // call, replayed while the call's arguments are unchanged
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux = nullptr;          // second stream of the forward transforms (plans made by cmif_plan_create*)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    // diagnostics (cmif_plan_set_wait_test): poll limit of the row kernel's bounded
    // waits (0: default) and an output row whose first bulk copy is withheld (-1: none)
    int test_wait_polls = 0;
    int test_withhold_row = -1;
    // Rotation angles per launch (CMIF_FLAG_BATCH_ANGLES, FP32 plans): up to ucap
    // angles run as units of one launch per stage; gcap is the geometry the FP32
    // workspace is sized for (ucap units; g itself when ucap = 1).
    int ucap = 1;
    Geom gcap{};
    int* maxn_u = nullptr;    // [ucap] per-unit max N of the gamma gate
    // CMIF_AUTO: per-pair precision (predicate up front, guard after the FP32 pass)
    Escal esc;
    double pred_scale = 0.0;   // kappa u log2(PQ): the predicate is pred_scale sqrt(|X_a| |Y_b|) >= pred_thr
    double pred_thr = 0.0;     // infinite when the predicate is off (CMIF_AUTO_PREDICATE=0)
};

namespace {

cmif_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return CMIF_OK;
    if (e == cudaErrorMemoryAllocation) return CMIF_ERR_OOM;
    return CMIF_ERR_CUDA;
}

// Row-kernel choice for precision T: the TMEM / TMA variant where it applies
// (FP32, Q = 512, 1024 or 2048), else B-marginals in shared memory when they fit,
// else in global memory.  Fills tm_cols, cb_smem and rows_grid.
template <typename T>
cmif_status choose_rows(cmif_plan p, Workspace<T>& w) {
    const Geom& g = p->gcap;  // the capacity geometry: the row grid serves every unit of a batched call
    int bps = 0;
    cudaError_t e = cudaSuccess;
    w.args.tm_cols = 0;
    const char* no_tm = std::getenv("CMIF_DISABLE_TMEM");
    if (sizeof(T) == 4 && !(no_tm && no_tm[0] == '1')) {
        const int cols = rows_tm_cols(g.Q, g.KB);
        if (cols > 0) {
            e = rows_tm_max_blocks_per_sm(g.Q, &bps);
            if (e != cudaSuccess) return from_cuda(e);
            if (bps >= 1) w.args.tm_cols = cols;
        }
    }
    if (w.args.tm_cols > 0) {
        // the TMEM kernel keeps the B-marginals in TMEM; calls that ask for the debug
        // count maps run the generic kernel, whose B-marginals may need the global slice
        w.cb_smem = !(p->flags & CMIF_FLAG_DEBUG_COUNTS) || rows_smem_bytes<T>(g.Q, g.KB, true) <= 200 * 1024;
    } else {
        const size_t smem_cb = rows_smem_bytes<T>(g.Q, g.KB, true);
        w.cb_smem = smem_cb <= 200 * 1024;
        e = rows_max_blocks_per_sm<T>(g.Q, g.KB, w.cb_smem, &bps);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (bps < 1) return CMIF_ERR_UNSUPPORTED;
    w.rows_grid = std::min(g.R, bps * p->num_sms);
    w.args.rows_grid = w.rows_grid;
    w.args.num_sms = p->num_sms;
    w.args.cb_smem = w.cb_smem;
    if (w.args.tm_cols > 0) {  // the generic kernel as an alternative the autotuner may pick
        w.tm_cols_avail = w.args.tm_cols;
        w.grid_tm = w.rows_grid;
        int bg = 0;
        if (rows_smem_bytes<T>(g.Q, g.KB, true) <= 200 * 1024 &&
            rows_max_blocks_per_sm<T>(g.Q, g.KB, true, &bg) == cudaSuccess && bg >= 1)
            w.grid_gen = std::min(g.R, bg * p->num_sms);
        cudaGetLastError();
    }
    return CMIF_OK;
}

// Switch an FP32 workspace between the TMEM and the generic row kernel (both
// prepared by choose_rows; the generic one only where its B-marginals fit in
// shared memory, so the workspace needs no global slice for it).
template <typename T>
bool set_rows_kernel(Workspace<T>& w, bool tmem) {
    if (tmem ? w.tm_cols_avail <= 0 : w.grid_gen <= 0) return false;
    w.args.tm_cols = tmem ? w.tm_cols_avail : 0;
    w.rows_grid = tmem ? w.grid_tm : w.grid_gen;
    w.args.rows_grid = w.rows_grid;
    if (!tmem) w.cb_smem = w.args.cb_smem = true;
    return true;
}

// Device bytes of the transform workspace of precision T (after choose_rows).
template <typename T>
size_t workspace_bytes(const Geom& g, const Workspace<T>& w) {
    const size_t cs = sizeof(cpx<T>);
    size_t off = 0;
    off = align_up(off + (size_t)g.KA * g.DA * g.HA * g.Qs * cs, 256);  // T1A
    off = align_up(off + (size_t)g.KB * g.DB * g.HB * g.Qs * cs, 256);  // T1B
    off = align_up(off + (size_t)g.KA * g.DA * g.Qh * g.P * cs, 256);   // FA
    off = align_up(off + (size_t)g.KB * g.DB * g.Qh * g.P * cs, 256);   // FB
    off = align_up(off + (size_t)(w.ypairs > 0 ? w.ypairs : g.KA * g.KB) * g.R * g.Qs * cs, 256);  // Y
    off = align_up(off + (w.cb_smem ? 0 : (size_t)w.rows_grid * g.KB * g.Q * sizeof(float)), 256);  // CB
    off = align_up(off + sizeof(int), 256);  // work counter
    if (w.rows_grid_w > 0) {
        off = align_up(off + (size_t)w.rows_grid_w * g.KB * g.Q * sizeof(double), 256);  // weighted B-marginals
        off = align_up(off + (size_t)g.R * g.C * sizeof(double), 256);                   // weighted N map
    }
    return off;
}

// Point the workspace's buffers into base (at least workspace_bytes long).
template <typename T>
void carve_workspace(const Geom& g, Workspace<T>& w, char* base) {
    const size_t cs = sizeof(cpx<T>);
    size_t off = 0;
    w.args.T1A = (cpx<T>*)(base + off); off = align_up(off + (size_t)g.KA * g.DA * g.HA * g.Qs * cs, 256);
    w.args.T1B = (cpx<T>*)(base + off); off = align_up(off + (size_t)g.KB * g.DB * g.HB * g.Qs * cs, 256);
    w.args.FA = (cpx<T>*)(base + off); off = align_up(off + (size_t)g.KA * g.DA * g.Qh * g.P * cs, 256);
    w.args.FB = (cpx<T>*)(base + off); off = align_up(off + (size_t)g.KB * g.DB * g.Qh * g.P * cs, 256);
    w.args.Y = (cpx<T>*)(base + off);
    off = align_up(off + (size_t)(w.ypairs > 0 ? w.ypairs : g.KA * g.KB) * g.R * g.Qs * cs, 256);
    w.args.cb_global = w.cb_smem ? nullptr : (float*)(base + off);
    off = align_up(off + (w.cb_smem ? 0 : (size_t)w.rows_grid * g.KB * g.Q * sizeof(float)), 256);
    w.args.work_ctr = (int*)(base + off);
    off = align_up(off + sizeof(int), 256);
    w.args.rows_grid_w = w.rows_grid_w;
    if (w.rows_grid_w > 0) {
        w.args.cbw = (double*)(base + off); off = align_up(off + (size_t)w.rows_grid_w * g.KB * g.Q * sizeof(double), 256);
        w.args.nw = (double*)(base + off);
    }
}

template <typename T>
cmif_status alloc_workspace(cmif_plan p, Workspace<T>& w) {
    cmif_status st = choose_rows<T>(p, w);
    if (st != CMIF_OK) return st;
    const size_t bytes = workspace_bytes<T>(p->g, w);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return CMIF_ERR_OOM; }
    w.base = base;
    w.bytes = bytes;
    carve_workspace<T>(p->g, w, (char*)base);
    return CMIF_OK;
}

void free_plan(cmif_plan p) {
    if (!p) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    if (p->mem) cudaFree(p->mem);
    if (p->stage) cudaFree(p->stage);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    p->prof.destroy();
    if (prev >= 0) cudaSetDevice(prev);
    delete p;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
void fill_io(PipeArgs<T>& a, const int32_t* A, const uint8_t* MA, const int32_t* B, const uint8_t* MB, double* mi,
             int32_t* n, int32_t* counts, DevStatus* st, const cmif_plan_s* p) {
    a.wait_polls = p->test_wait_polls;
    a.withhold_row = p->test_withhold_row;
    a.aux = p->aux;
    a.ev_fork = p->ev_fork;
    a.ev_join = p->ev_join;
    a.A = A;
    a.MA = MA;
    a.B = B;
    a.MB = MB;
    a.mi = mi;
    a.n = n;
    a.counts = counts;
    a.st = st;
}

// Alg. 1's search window (Sec. 3.6: A zero-padded by ceil(|X_B|_i (1 - gamma)) along
// each axis; X_S = the shifts that keep B's domain inside padded A's):
//   chi_i in [|X_B|_i - |X_A|_i - p_i, p_i], intersected with the full range.
// In output indices (row = chi_y + H_A - 1) that is [H_B - 1 - p_y, H_A - 1 + p_y].
// Without CMIF_FLAG_WINDOW the window is the whole map.  Returns false when the
// window is empty (B cannot fit inside padded A).
bool call_geom(const cmif_plan p, double gamma, Geom* out) {
    Geom g = p->g;
    if (p->flags & CMIF_FLAG_WINDOW) {
        const int py = (int)std::ceil(g.HB * (1.0 - gamma)), px = (int)std::ceil(g.WB * (1.0 - gamma));
        g.r0 = std::max(0, g.HB - 1 - py);
        g.r1 = std::min(g.R, g.HA + py);
        g.c0 = std::max(0, g.WB - 1 - px);
        g.c1 = std::min(g.C, g.WA + px);
    }
    *out = g;
    return g.r0 < g.r1 && g.c0 < g.c1;
}

// Second precision for one stage of the pair list (entries [lrange[0], lrange[1])):
// the level-set transforms of the planes the listed pairs need, then, chunk by
// chunk, their products, inverse column transforms and exact counts (into the
// plan's ov buffer).  Every launch returns at once when the stage lists nothing.
template <typename T>
cudaError_t tier2_stage(cmif_plan p, Workspace<T>& w, const Geom& g, const int32_t* A, const uint8_t* MA,
                        const int32_t* B, const uint8_t* MB, const int* lrange, cudaStream_t s) {
    PipeArgs<T> b = w.args;
    fill_io(b, A, MA, B, MB, nullptr, nullptr, nullptr, p->st, p);
    b.prof = p->prof.enabled ? &p->prof : nullptr;
    b.prec_slot = 1;
    b.conditional = 0;
    b.needA = p->esc.needA;
    b.needB = p->esc.needB;
    b.stages = STAGE_FWD_A | STAGE_FWD_B;
    cudaError_t e = run_pipeline<T>(g, b, s);
    if (e != cudaSuccess) return e;
    b.needA = b.needB = nullptr;
    b.plist = p->esc.plist;
    b.lrange = lrange;
    b.ov = p->esc.ov;
    b.chunk_cap = p->esc.chunk;
    for (int off = 0; off < p->esc.cap; off += p->esc.chunk) {
        b.chunk_off = off;
        e = run_pair_counts<T>(g, b, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename Fn>
cudaError_t with_tier2(cmif_plan p, Fn&& fn) {
    return p->tier2 == CMIF_FP64 ? fn(p->w64) : fn(p->ws32);
}

// CMIF_AUTO: FP32 transforms with per-pair precision.  The predicate picks the
// pairs whose FP32 correlation would not round exactly and computes them in the
// second precision first; the FP32 row pass takes their exact counts and records
// every other pair's residual; pairs that still breach the guard are computed in
// the second precision too and the FP32 row pass runs once more (on the device,
// only after a breach).  Counts of every pair are then exact (Sec. 3.2).
cmif_status compute_map_auto(cmif_plan p, const Geom& g, const int32_t* A, const uint8_t* MA, const int32_t* B,
                             const uint8_t* MB, double* mi, int32_t* n, int32_t* counts, cudaStream_t s,
                             unsigned stages32) {
    Escal& E = p->esc;
    cudaError_t e = cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s);
    PipeArgs<float> a = p->w32.args;
    fill_io(a, A, MA, B, MB, mi, n, counts, p->st, p);
    a.prof = p->prof.enabled ? &p->prof : nullptr;
    a.prec_slot = 0;
    a.conditional = 0;
    // 1. FP32 level-set transforms, with the label pixel counts of the predicate
    if (e == cudaSuccess && (stages32 & STAGE_FWD_A)) e = cudaMemsetAsync(E.popA, 0, g.KA * sizeof(int), s);
    if (e == cudaSuccess && (stages32 & STAGE_FWD_B)) e = cudaMemsetAsync(E.popB, 0, g.KB * sizeof(int), s);
    if (e != cudaSuccess) return from_cuda(e);
    a.popA = (stages32 & STAGE_FWD_A) ? E.popA : nullptr;
    a.popB = (stages32 & STAGE_FWD_B) ? E.popB : nullptr;
    a.stages = stages32 & (STAGE_FWD_A | STAGE_FWD_B);
    if (a.stages) e = run_pipeline<float>(g, a, s);
    a.popA = a.popB = nullptr;
    // 2. the predicate: stage 1 of the list
    p->prof.begin("select_pairs", s);
    if (e == cudaSuccess)
        e = launch_select_pairs(E.popA, E.popB, g.KA, g.KB, p->pred_scale, p->pred_thr, E.cap, E.plist, E.hdr,
                                E.ov_slot, E.pair_res, E.needA, E.needB, p->st, s);
    p->prof.end(s);
    // 3. second precision for the predicted pairs
    if (e == cudaSuccess)
        e = with_tier2(p, [&](auto& w) { return tier2_stage(p, w, g, A, MA, B, MB, E.hdr + 0, s); });
    // 4. FP32 pair stages; listed pairs take their exact counts, the others' residuals are kept per pair
    a.ov = E.ov;
    a.ov_slot = E.ov_slot;
    a.pair_res = E.pair_res;
    a.stages = stages32 & STAGE_PAIRS;
    if (e == cudaSuccess) e = run_pipeline<float>(g, a, s);
    // 5. the guard: breached pairs form stage 2 of the list
    p->prof.begin("check_pairs", s);
    if (e == cudaSuccess)
        e = launch_check_pairs(E.pair_res, g.KA, g.KB, E.cap, E.plist, E.hdr, E.ov_slot, E.needA, E.needB, p->st, s);
    p->prof.end(s);
    // 6. second precision for them, 7. the FP32 row pass again (only after a breach)
    if (e == cudaSuccess)
        e = with_tier2(p, [&](auto& w) { return tier2_stage(p, w, g, A, MA, B, MB, E.hdr + 1, s); });
    a.stages = STAGE_ROWS;
    a.conditional = 1;
    if (e == cudaSuccess) e = run_pipeline<float>(g, a, s);
    if (e != cudaSuccess) return from_cuda(e);
    p->prof.begin("finalize", s);
    e = launch_finalize(p->st, 2, 2, s);
    if (e == cudaSuccess) e = launch_merge_status(p->st, p->st_total, 2, s);
    p->prof.end(s);
    return from_cuda(e);
}

// One full map into (mi, n, counts); its status in p->st (reset here) is folded
// into p->st_total.  stages32 selects the FP32 stages (A's transforms may be
// reused across calls); an FP64 or two-term pass always recomputes everything.
cmif_status compute_map(cmif_plan p, const Geom& g, const int32_t* A, const uint8_t* MA, const int32_t* B,
                        const uint8_t* MB, double* mi, int32_t* n, int32_t* counts, cudaStream_t s,
                        unsigned stages32 = STAGE_ALL) {
    if (p->prec == CMIF_AUTO) return compute_map_auto(p, g, A, MA, B, MB, mi, n, counts, s, stages32);
    cudaError_t e = cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return from_cuda(e);
    if (p->prec == CMIF_FP32) {
        PipeArgs<float> a = p->w32.args;
        fill_io(a, A, MA, B, MB, mi, n, counts, p->st, p);
        a.prof = p->prof.enabled ? &p->prof : nullptr;
        a.stages = stages32;
        a.prec_slot = 0;
        a.conditional = 0;
        e = run_pipeline<float>(g, a, s);
    } else if (p->prec == CMIF_FP64) {
        PipeArgs<double> a = p->w64.args;
        fill_io(a, A, MA, B, MB, mi, n, counts, p->st, p);
        a.prof = p->prof.enabled ? &p->prof : nullptr;
        a.stages = STAGE_ALL;
        a.prec_slot = 1;
        a.conditional = 0;
        e = run_pipeline<double>(g, a, s);
    } else {
        PipeArgs<df32> a = p->ws32.args;
        fill_io(a, A, MA, B, MB, mi, n, counts, p->st, p);
        a.prof = p->prof.enabled ? &p->prof : nullptr;
        a.stages = STAGE_ALL;
        a.prec_slot = 1;
        a.conditional = 0;
        e = run_pipeline<df32>(g, a, s);
    }
    if (e != cudaSuccess) return from_cuda(e);
    const int slot_default = (p->prec == CMIF_FP64 || p->prec == CMIF_SPLIT32) ? 1 : 0;
    p->prof.begin("finalize", s);
    e = launch_finalize(p->st, slot_default, slot_default, s);
    if (e == cudaSuccess) e = launch_merge_status(p->st, p->st_total, slot_default, s);
    p->prof.end(s);
    return from_cuda(e);
}

// Validate sizes and flags, set the geometry, pick kernels; allocates nothing
// (except the per-device twiddle tables on first use).
cmif_status plan_init(cmif_plan p, int H_A, int W_A, int H_B, int W_B, int K_A, int K_B, cmif_precision prec,
                      unsigned flags, int D_A = 1, int D_B = 1, int max_units = kMaxUnits) {
    if (H_A < 1 || W_A < 1 || H_B < 1 || W_B < 1 || K_A < 1 || K_B < 1 || K_A > 64 || K_B > 64)
        return CMIF_ERR_INVALID_ARG;
    if (D_A < 1 || D_B < 1 || D_A > 1024 || D_B > 1024) return CMIF_ERR_INVALID_ARG;
    if ((long long)D_A * H_A * W_A > (1LL << 22) || (long long)D_B * H_B * W_B > (1LL << 22))
        return CMIF_ERR_INVALID_ARG;
    const bool volume = D_A > 1 || D_B > 1;
    if (volume && (flags & (CMIF_FLAG_WINDOW | CMIF_FLAG_WEIGHTED))) return CMIF_ERR_UNSUPPORTED;
    if (flags & ~(CMIF_FLAG_DEBUG_COUNTS | CMIF_FLAG_GRAPH | CMIF_FLAG_WINDOW | CMIF_FLAG_NMI | CMIF_FLAG_WEIGHTED |
                  CMIF_FLAG_AUTOTUNE | CMIF_FLAG_BATCH_ANGLES))
        return CMIF_ERR_INVALID_ARG;
    // weighted maps: FP64 transforms (real counts, no rounding), MI only
    if ((flags & CMIF_FLAG_WEIGHTED) && (prec != CMIF_FP64 || (flags & (CMIF_FLAG_NMI | CMIF_FLAG_DEBUG_COUNTS))))
        return CMIF_ERR_UNSUPPORTED;
    if (prec != CMIF_FP32 && prec != CMIF_SPLIT32 && prec != CMIF_FP64 && prec != CMIF_AUTO) return CMIF_ERR_INVALID_ARG;
    Geom g{};
    g.HA = H_A; g.WA = W_A; g.HB = H_B; g.WB = W_B; g.KA = K_A; g.KB = K_B;
    g.DA = D_A; g.DB = D_B; g.Dz = D_A + D_B - 1; g.units = 1;
    g.R2 = H_A + H_B - 1;
    g.R = g.Dz * g.R2;
    g.C = W_A + W_B - 1;
    // FP32 plans may take lengths 3 * 2^k (the two-term and FP64 kernels, and hence
    // AUTO's second precision, exist for powers of two only)
    const char* p2e = std::getenv("CMIF_POW2_ONLY");
    const bool mixed = prec == CMIF_FP32 && !(p2e && p2e[0] == '1');
    g.P = transform_size(g.R2, mixed);
    g.Q = transform_size(g.C, mixed);
    {
        // The row transform prefers the widths of the Tensor-Memory row kernel (512,
        // 1024, 2048) to a shorter 3 * 2^k: that kernel turns out counts about twice as
        // fast as the generic one, which outweighs the 4/3 more points of the longer
        // rows (and of the pair-column transforms over their columns).  Plans that ask
        // for the count maps run the generic kernel and keep the shorter width.
        const char* tq = std::getenv("CMIF_ROWS_POW2");  // "0": keep the shortest width
        const char* no_tm = std::getenv("CMIF_DISABLE_TMEM");
        const int q2 = transform_size(g.C, false);
        if (mixed && q2 != g.Q && (q2 == 512 || q2 == 1024 || q2 == 2048) && !(tq && tq[0] == '0') &&
            !(no_tm && no_tm[0] == '1') && !(flags & CMIF_FLAG_DEBUG_COUNTS) && rows_tm_cols(q2, K_B) > 0)
            g.Q = q2;
    }
    if (g.P > 4096 || g.Q > 4096) return CMIF_ERR_UNSUPPORTED;
    g.Qh = g.Q / 2 + 1;
    g.Qs = (int)align_up((size_t)g.Qh, 4);
    g.r0 = 0; g.r1 = g.R; g.c0 = 0; g.c1 = g.C;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return CMIF_ERR_CUDA;
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return CMIF_ERR_CUDA;
    p->g = g;
    p->gcap = g;
    p->ucap = 1;
    if ((flags & CMIF_FLAG_BATCH_ANGLES) && !volume && prec == CMIF_FP32) {
        // as many angles per launch as 40% of the free device memory holds (at most 64)
        const size_t per_unit = (size_t)K_B * H_B * g.Qs * 8 + (size_t)K_B * g.Qh * g.P * 8 +
                                (size_t)K_A * K_B * g.R * g.Qs * 8 + (size_t)g.R * g.C * 12 + (size_t)H_B * W_B * 5;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return CMIF_ERR_CUDA;
        long long u = (long long)(0.4 * (double)fr / (double)per_unit);
        const char* ue = std::getenv("CMIF_ANGLE_BATCH");  // an upper bound on the units per launch
        if (ue && std::atoi(ue) > 0) u = std::min<long long>(u, std::atoi(ue));
        p->ucap = (int)std::max<long long>(1, std::min<long long>(u, std::min(max_units, kMaxUnits)));
        if (p->ucap > 1) {
            p->gcap.units = p->ucap;
            p->gcap.DB = p->ucap;
            p->gcap.R = p->ucap * g.R2;
        }
    }
    p->prec = prec;
    p->flags = flags;
    p->use_graph = (flags & CMIF_FLAG_GRAPH) != 0;
    const char* t2 = std::getenv("CMIF_AUTO_TIER2");  // "fp64" makes AUTO re-run in FP64 instead of split FP32
    p->tier2 = (t2 && std::strcmp(t2, "fp64") == 0) ? CMIF_FP64 : CMIF_SPLIT32;
    cmif_status st = CMIF_OK;
    if (prec == CMIF_FP32 || prec == CMIF_AUTO) {
        st = choose_rows<float>(p, p->w32);
        p->has32 = (st == CMIF_OK);
    }
    if (st == CMIF_OK && (prec == CMIF_FP64 || (prec == CMIF_AUTO && p->tier2 == CMIF_FP64))) {
        st = choose_rows<double>(p, p->w64);
        p->has64 = (st == CMIF_OK);
        if (st == CMIF_OK && (flags & CMIF_FLAG_WEIGHTED)) {
            int bps = 0;
            if (rows_w_max_blocks_per_sm(g.Q, &bps) != cudaSuccess) return CMIF_ERR_CUDA;
            if (bps < 1) return CMIF_ERR_UNSUPPORTED;
            p->w64.rows_grid_w = std::min(g.R, bps * p->num_sms);
        }
    }
    if (st == CMIF_OK && (prec == CMIF_SPLIT32 || (prec == CMIF_AUTO && p->tier2 == CMIF_SPLIT32))) {
        st = choose_rows<df32>(p, p->ws32);
    }
    if (st != CMIF_OK) return st;
    if (prec == CMIF_AUTO) {
        // per-pair precision: the second precision holds the products of one chunk
        // of listed pairs at a time (a few GB at most), and the exact counts of at
        // most `cap` listed pairs
        const int npairs = K_A * K_B;
        const size_t per_pair = (size_t)g.R * g.Qs * (p->tier2 == CMIF_FP64 ? sizeof(cpx<double>) : sizeof(cpx<df32>));
        const size_t budget = 4ull << 30;
        p->esc.chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)npairs, budget / per_pair));
        p->esc.cap = std::min(npairs, 128);
        if (p->tier2 == CMIF_FP64) p->w64.ypairs = p->esc.chunk;
        else p->ws32.ypairs = p->esc.chunk;
        // the predicate: an FFT correlation of two 0/1 planes errs by about
        // kappa u log2(PQ) sqrt(|X_a| |Y_b|) (u = 2^-24); kappa = 0.25 bounds the
        // residuals measured at 256^2 and 1024^2 with balanced labels (1024^2, K = 16:
        // 0.0195 at |X| ~ 2^16, where the model gives 0.021); pairs whose estimate
        // reaches half the 0.25 guard go to the second precision up front
        const double logpq = std::log2((double)g.P * (double)g.Q * (double)std::max(D_A, D_B));
        p->pred_scale = 0.25 * std::ldexp(1.0, -24) * logpq;
        const char* pe = std::getenv("CMIF_AUTO_PREDICATE");  // "0": off; "all": every pair (diagnostics)
        p->pred_thr = (pe && std::strcmp(pe, "0") == 0) ? HUGE_VAL
                    : (pe && std::strcmp(pe, "all") == 0) ? 0.0 : 0.5 * (double)kResidualGuard;
    }
    const char* cm_env = std::getenv("CMIF_COL_M");  // column-team variant of the FP32 transforms
    p->w32.args.col_m = (cm_env && std::strcmp(cm_env, "16") == 0) ? 16 : 0;
    const int nmi = (flags & CMIF_FLAG_NMI) ? 1 : 0;
    p->w32.args.nmi = nmi;
    p->w64.args.nmi = nmi;
    p->ws32.args.nmi = nmi;
    Tw<float> tf;
    Tw<double> td;
    Tw<df32> ts;
    e = get_twiddles(p->device, &tf, &td, &ts);
    if (e != cudaSuccess) return from_cuda(e);
    p->w32.args.tw = tf;
    p->w64.args.tw = td;
    p->ws32.args.tw = ts;
    p->nparts = 2 * p->num_sms;
    return CMIF_OK;
}

size_t small_bytes_of(const cmif_plan p) {
    const Geom& g = p->g;
    const size_t u = (size_t)p->ucap;
    size_t off = align_up(sizeof(DevStatus), 256) * 2;
    off = align_up(off + u * p->nparts * sizeof(PeakPart), 256);
    off = align_up(off + u * g.R * g.C * sizeof(int32_t), 256);
    off = align_up(off + u * g.R * g.C * sizeof(double), 256);
    off = align_up(off + u * g.HB * g.WB * sizeof(int32_t), 256);
    off = align_up(off + u * g.HB * g.WB, 256);
    off = align_up(off + (size_t)(kMaxAngles + 2) * sizeof(PeakRec), 256);
    off = align_up(off + u * sizeof(int), 256);
    return off;
}

// Device bytes of everything the plan uses: small buffers + one workspace per precision.
// Device bytes of the per-pair precision buffers (CMIF_AUTO plans).
size_t esc_bytes(const cmif_plan p) {
    if (p->prec != CMIF_AUTO) return 0;
    const Geom& g = p->g;
    const size_t np = (size_t)g.KA * g.KB;
    size_t off = 0;
    off = align_up(off + g.KA * sizeof(int), 256) + align_up(g.KB * sizeof(int), 256);
    off += align_up(g.KA, 256) + align_up(g.KB, 256);
    off += align_up(np * sizeof(int), 256) + 256 + align_up(np * sizeof(int), 256) + align_up(np * sizeof(unsigned), 256);
    off += align_up((size_t)p->esc.cap * g.R * g.Q * sizeof(int32_t), 256);
    return off;
}

void esc_carve(cmif_plan p, char* base) {
    const Geom& g = p->g;
    const size_t np = (size_t)g.KA * g.KB;
    size_t off = 0;
    Escal& E = p->esc;
    E.popA = (int*)(base + off); off += align_up(g.KA * sizeof(int), 256);
    E.popB = (int*)(base + off); off += align_up(g.KB * sizeof(int), 256);
    E.needA = (unsigned char*)(base + off); off += align_up(g.KA, 256);
    E.needB = (unsigned char*)(base + off); off += align_up(g.KB, 256);
    E.plist = (int*)(base + off); off += align_up(np * sizeof(int), 256);
    E.hdr = (int*)(base + off); off += 256;
    E.ov_slot = (int*)(base + off); off += align_up(np * sizeof(int), 256);
    E.pair_res = (unsigned*)(base + off); off += align_up(np * sizeof(unsigned), 256);
    E.ov = (int32_t*)(base + off); off += align_up((size_t)E.cap * g.R * g.Q * sizeof(int32_t), 256);
    E.bytes = off;
}

size_t plan_bytes(cmif_plan p) {
    size_t b = small_bytes_of(p) + esc_bytes(p);
    if (p->has32) b += workspace_bytes<float>(p->gcap, p->w32);
    if (p->has64) b += workspace_bytes<double>(p->g, p->w64);
    if (p->ws32.rows_grid > 0) b += workspace_bytes<df32>(p->g, p->ws32);
    return b;
}

// Point the plan's buffers into base (plan_bytes long) and clear its status words.
cmif_status plan_carve(cmif_plan p, char* base) {
    const Geom& g = p->g;
    size_t off = 0;
    p->st = (DevStatus*)(base + off); off += align_up(sizeof(DevStatus), 256);
    p->st_total = (DevStatus*)(base + off); off += align_up(sizeof(DevStatus), 256);
    const size_t u = (size_t)p->ucap;
    p->parts = (PeakPart*)(base + off); off = align_up(off + u * p->nparts * sizeof(PeakPart), 256);
    p->nbuf = (int32_t*)(base + off); off = align_up(off + u * g.R * g.C * sizeof(int32_t), 256);
    p->mibuf = (double*)(base + off); off = align_up(off + u * g.R * g.C * sizeof(double), 256);
    p->wB = (int32_t*)(base + off); off = align_up(off + u * g.HB * g.WB * sizeof(int32_t), 256);
    p->wM = (uint8_t*)(base + off); off = align_up(off + u * g.HB * g.WB, 256);
    p->peaks = base + off; off = align_up(off + (size_t)(kMaxAngles + 2) * sizeof(PeakRec), 256);
    p->maxn_u = (int*)(base + off); off = align_up(off + u * sizeof(int), 256);
    p->small_bytes = off;
    if (p->has32) {
        carve_workspace<float>(p->gcap, p->w32, base + off);
        off += workspace_bytes<float>(p->gcap, p->w32);
    }
    if (p->has64) { carve_workspace<double>(g, p->w64, base + off); off += workspace_bytes<double>(g, p->w64); }
    if (p->ws32.rows_grid > 0) { carve_workspace<df32>(g, p->ws32, base + off); off += workspace_bytes<df32>(g, p->ws32); }
    if (p->prec == CMIF_AUTO) { esc_carve(p, base + off); off += p->esc.bytes; }
    p->w32.bytes = p->has32 ? workspace_bytes<float>(p->gcap, p->w32) : 0;
    p->w64.bytes = p->has64 ? workspace_bytes<double>(g, p->w64) : 0;
    p->ws32.bytes = p->ws32.rows_grid > 0 ? workspace_bytes<df32>(g, p->ws32) : 0;
    if (cudaMemset(p->st, 0, 2 * align_up(sizeof(DevStatus), 256)) != cudaSuccess) return CMIF_ERR_CUDA;
    return CMIF_OK;
}

template <typename V>
void key_add(std::vector<unsigned char>& k, const V& v) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), b, b + sizeof(V));
}

// Run `record` (which enqueues a call's launches on the stream it is given)
// directly, or -- with graph replay on -- capture it once into a CUDA graph on
// the plan's own stream and replay the graph on s while the call's key (its
// arguments) is unchanged.  Capture uses relaxed mode and a non-default
// stream, so the caller's stream may be the legacy default stream.
template <typename Fn>
cmif_status run_graph(cmif_plan p, cudaStream_t s, std::vector<unsigned char> key, Fn&& record) {
    if (!p->use_graph) return record(s);
    key_add(key, p->test_wait_polls);  // baked into the captured launches
    key_add(key, p->test_withhold_row);
    cudaError_t e = cudaSuccess;
    if (!(p->gexec && key == p->gkey)) {
        if (!p->cap_stream) {
            e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return from_cuda(e);
        }
        if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
        const bool prof = p->prof.enabled;
        p->prof.enabled = false;  // no per-launch events inside a graph
        e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { p->prof.enabled = prof; return from_cuda(e); }
        cmif_status st = record(p->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &graph);
        p->prof.enabled = prof;
        if (st != CMIF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaGraphInstantiate(&p->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { p->gexec = nullptr; return from_cuda(e); }
        p->gkey = key;
    }
    p->prof.begin("graph", s);
    e = cudaGraphLaunch(p->gexec, s);
    p->prof.end(s);
    return from_cuda(e);
}

// Alg. 1 over rotations with up to ucap angles per launch of every stage: A's
// transforms once, then per chunk of angles one warp launch, B's row and column
// transforms of all the chunk's rotated images, one pair-column and one row
// launch over (angle, pair) and (angle, row) work, and the per-angle peaks.
cmif_status align_core_units(cmif_plan plan, const Geom& g, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                             const uint8_t* M_B, const double* angles, int n_angles, double gamma, int top_k,
                             void* topk_dev, double* mi_maps, int32_t* n_maps, cudaStream_t s) {
    const size_t RC = (size_t)g.R * g.C;
    PeakRec* peaks = reinterpret_cast<PeakRec*>(plan->peaks);
    cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return from_cuda(e);
    PipeArgs<float> a = plan->w32.args;
    fill_io(a, A, M_A, nullptr, nullptr, nullptr, nullptr, nullptr, plan->st, plan);
    a.prof = plan->prof.enabled ? &plan->prof : nullptr;
    a.prec_slot = 0;
    a.conditional = 0;
    a.stages = STAGE_FWD_A;
    e = run_pipeline<float>(g, a, s);  // A's transforms, shared by every angle
    if (e != cudaSuccess) return from_cuda(e);
    for (int c0 = 0; c0 < n_angles; c0 += plan->ucap) {
        const int G = std::min(plan->ucap, n_angles - c0);
        Geom gu = g;
        gu.units = G;
        gu.DB = G;
        gu.R = G * g.R2;
        double* mi = mi_maps ? mi_maps + (size_t)c0 * RC : plan->mibuf;
        int32_t* nm = n_maps ? n_maps + (size_t)c0 * RC : plan->nbuf;
        if (g.r0 > 0 || g.r1 < g.R) {  // rows outside the window are not computed: zero
            if (mi_maps) e = cudaMemsetAsync(mi, 0, G * RC * sizeof(double), s);
            if (e == cudaSuccess && n_maps) e = cudaMemsetAsync(nm, 0, G * RC * sizeof(int32_t), s);
            if (e != cudaSuccess) return from_cuda(e);
        }
        plan->prof.begin("warp_nn", s);
        e = launch_warp_nn_multi(B, M_B, g.HB, g.WB, angles + c0, G, plan->wB, plan->wM, s);
        plan->prof.end(s);
        if (e == cudaSuccess) e = cudaMemsetAsync(plan->st, 0, sizeof(DevStatus), s);
        if (e != cudaSuccess) return from_cuda(e);
        fill_io(a, A, M_A, plan->wB, plan->wM, mi, nm, nullptr, plan->st, plan);
        a.stages = STAGE_FWD_B | STAGE_PAIRS;
        a.rows_grid = std::min(G * (g.r1 - g.r0), plan->w32.rows_grid);
        e = run_pipeline<float>(gu, a, s);
        if (e != cudaSuccess) return from_cuda(e);
        plan->prof.begin("finalize", s);
        e = launch_finalize(plan->st, 0, 0, s);
        if (e == cudaSuccess) e = launch_merge_status(plan->st, plan->st_total, 0, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
        plan->prof.begin("peak", s);
        e = launch_peak_units(mi, nm, gu, plan->st, gamma, plan->parts, plan->nparts, c0, peaks + c0, plan->maxn_u, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    plan->prof.begin("topk", s);
    e = launch_topk(peaks, n_angles, top_k, topk_dev, s);
    plan->prof.end(s);
    return from_cuda(e);
}

// Alg. 1 over rotations for one pair (see cmif_align_rotations); enqueues on s.
cmif_status align_core(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B, const uint8_t* M_B,
                       const double* angles, int n_angles, double gamma, int top_k, void* topk_dev, double* mi_maps,
                       int32_t* n_maps, cudaStream_t s) {
    Geom g;
    if (!call_geom(plan, gamma, &g)) return CMIF_ERR_INVALID_ARG;
    if (plan->ucap > 1 && plan->prec == CMIF_FP32)
        return align_core_units(plan, g, A, M_A, B, M_B, angles, n_angles, gamma, top_k, topk_dev, mi_maps, n_maps, s);
    const size_t RC = (size_t)g.R * g.C;
    cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return from_cuda(e);
    PeakRec* peaks = reinterpret_cast<PeakRec*>(plan->peaks);
    for (int i = 0; i < n_angles; ++i) {
        plan->prof.begin("warp_nn", s);
        e = launch_warp_nn(B, M_B, g.HB, g.WB, angles[i], plan->wB, plan->wM, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
        double* mi = mi_maps ? mi_maps + (size_t)i * RC : plan->mibuf;
        int32_t* nm = n_maps ? n_maps + (size_t)i * RC : plan->nbuf;
        if (g.r0 > 0 || g.r1 < g.R) {  // rows outside the window are not computed: zero
            if (mi_maps) e = cudaMemsetAsync(mi, 0, RC * sizeof(double), s);
            if (e == cudaSuccess && n_maps) e = cudaMemsetAsync(nm, 0, RC * sizeof(int32_t), s);
            if (e != cudaSuccess) return from_cuda(e);
        }
        const unsigned stages = (i == 0) ? STAGE_ALL : (STAGE_FWD_B | STAGE_PAIRS);
        cmif_status cs = compute_map(plan, g, A, M_A, plan->wB, plan->wM, mi, nm, nullptr, s, stages);
        if (cs != CMIF_OK) return cs;
        plan->prof.begin("peak", s);
        e = launch_peak(mi, nm, g, plan->st, gamma, plan->parts, plan->nparts, i, peaks + i, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    plan->prof.begin("topk", s);
    e = launch_topk(peaks, n_angles, top_k, topk_dev, s);
    plan->prof.end(s);
    return from_cuda(e);
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Autotuner: the FP32 path of a plan has a few launch-shape choices whose best
// value depends on the transform sizes, the label counts and the GPU: the
// column transforms' lanes per group (32, or 16 with a radix-R exchange), the
// row kernel (Tensor-Memory or generic) and the pair-column kernel's persistent
// blocks per SM.  The tuner times every candidate on synthetic labels of the
// plan's sizes (CUDA events, the median of a few maps) and keeps the fastest;
// results are cached per process and, optionally, in a JSON-lines file keyed
// on (P, Q, K_A, K_B, depths, precision, SM count, device name).

struct TuneRec {
    int col_m = 0, tmem = 0, cols_bps = 0;
    double ms = 0.0;
};

std::string tune_key(const cmif_plan p) {
    const Geom& g = p->g;
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, p->device);
    char buf[128];
    std::snprintf(buf, sizeof buf, "P%d.Q%d.KA%d.KB%d.DA%d.DB%d.%s.sm%d.", g.P, g.Q, g.KA, g.KB, g.DA, g.DB,
                  p->prec == CMIF_AUTO ? "auto" : "fp32", p->num_sms);
    return std::string(buf) + std::string(prop.name, strnlen(prop.name, sizeof prop.name));
}

std::mutex g_tune_mu;
std::map<std::string, TuneRec> g_tune_cache;

int json_int(const std::string& line, const char* field, int dflt) {
    const std::string pat = std::string("\"") + field + "\": ";
    const size_t at = line.find(pat);
    return at == std::string::npos ? dflt : std::atoi(line.c_str() + at + pat.size());
}

bool tune_lookup_file(const char* path, const std::string& key, TuneRec* out) {
    if (!path) return false;
    std::FILE* f = std::fopen(path, "r");
    if (!f) return false;
    bool found = false;
    char line[1024];
    const std::string kpat = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof line, f)) {
        const std::string l(line);
        if (l.find(kpat) == std::string::npos) continue;  // the last matching line wins
        out->col_m = json_int(l, "col_m", 0);
        out->tmem = json_int(l, "tmem_rows", 0);
        out->cols_bps = json_int(l, "cols_blocks_per_sm", 0);
        const size_t at = l.find("\"ms\": ");
        out->ms = at == std::string::npos ? 0.0 : std::atof(l.c_str() + at + 6);
        found = true;
    }
    std::fclose(f);
    return found;
}

void tune_store_file(const char* path, const std::string& key, const TuneRec& r) {
    if (!path) return;
    std::FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"col_m\": %d, \"tmem_rows\": %d, \"cols_blocks_per_sm\": %d, \"ms\": %.4f}\n",
                 key.c_str(), r.col_m, r.tmem, r.cols_bps, r.ms);
    std::fclose(f);
}

void apply_tune(cmif_plan p, const TuneRec& r) {
    p->w32.args.col_m = r.col_m;
    p->w32.args.cols_bps = r.cols_bps;
    set_rows_kernel(p->w32, r.tmem != 0);
    if (p->gexec) {  // captured launches used the old shapes
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
        p->gkey.clear();
    }
}

cmif_status autotune(cmif_plan p, const char* cache_path, cmif_tuning* out) {
    if (!p->has32) {  // FP64 / two-term plans: nothing to choose
        if (out) *out = cmif_tuning{0, 0, 0, 0.0, 0, 0};
        return CMIF_OK;
    }
    const std::string key = tune_key(p);
    TuneRec best;
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { best = it->second; have = true; }
    }
    int from_cache = have ? 1 : 0;
    if (!have && tune_lookup_file(cache_path, key, &best)) { have = true; from_cache = 2; }
    int ncand = 0;
    if (!have) {
        const Geom& g = p->g;
        const long long nA = (long long)g.DA * g.HA * g.WA, nB = (long long)g.DB * g.HB * g.WB;
        int32_t* lab = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaMalloc(&lab, (size_t)(nA + nB) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = launch_fill_labels(lab, nA, g.KA, 12345u, s);
        if (e == cudaSuccess) e = launch_fill_labels(lab + nA, nB, g.KB, 67890u, s);
        std::vector<TuneRec> cands;
        const int col_ms[2] = {0, 16};
        for (int cm : col_ms) {
            if (cm == 16 && g.P < 1024) continue;
            for (int tm = 1; tm >= 0; --tm) {
                if (tm ? p->w32.tm_cols_avail <= 0 : (p->w32.tm_cols_avail > 0 && p->w32.grid_gen <= 0)) continue;
                for (int bps : {0, 1}) cands.push_back(TuneRec{cm, tm, bps, 0.0});
            }
        }
        const TuneRec before{p->w32.args.col_m, p->w32.args.tm_cols > 0 ? 1 : 0, p->w32.args.cols_bps, 0.0};
        double best_ms = 1e30;
        for (TuneRec& c : cands) {
            if (e != cudaSuccess) break;
            apply_tune(p, c);
            PipeArgs<float> a = p->w32.args;
            fill_io(a, lab, nullptr, lab + nA, nullptr, p->mibuf, p->nbuf, nullptr, p->st, p);
            a.stages = STAGE_ALL;
            a.prec_slot = 0;
            a.conditional = 0;
            std::vector<float> ts;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = run_pipeline<float>(g, a, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ts.push_back(ms);  // the first run warms up
            }
            if (e != cudaSuccess) break;
            std::sort(ts.begin(), ts.end());
            c.ms = ts[ts.size() / 2];
            ++ncand;
            if (c.ms < best_ms) { best_ms = c.ms; best = c; }
        }
        if (s) cudaStreamDestroy(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (lab) cudaFree(lab);
        if (e != cudaSuccess) {
            apply_tune(p, before);
            cudaGetLastError();
            return from_cuda(e);
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
        tune_store_file(cache_path, key, best);
    } else if (from_cache == 2) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    // a cached choice may name an alternative this plan lacks (other flags): fall back
    if (best.tmem ? p->w32.tm_cols_avail <= 0 : (p->w32.tm_cols_avail > 0 && p->w32.grid_gen <= 0)) best.tmem = !best.tmem;
    if (best.col_m == 16 && p->g.P < 1024) best.col_m = 0;
    apply_tune(p, best);
    if (out) *out = cmif_tuning{best.col_m ? best.col_m : 32, best.tmem, best.cols_bps, best.ms, from_cache, ncand};
    return CMIF_OK;
}

}  // namespace

struct cmif_batch_s {
    int device = 0;
    std::vector<cmif_pair_desc> descs;
    std::vector<std::vector<double>> angles;
    std::vector<cmif_plan> plans;  // per pair, all carved from mem
    void* mem = nullptr;
    size_t mem_bytes = 0;
    DevStatus* total = nullptr;    // status of the whole batch
    cmif_plan_s graph_holder;      // capture stream / graph of the batch
    cudaStream_t last_stream = nullptr;
    std::vector<unsigned char> gkey;
};

extern "C" {

namespace {
cmif_status plan_create(cmif_plan* out, int D_A, int H_A, int W_A, int D_B, int H_B, int W_B, int K_A, int K_B,
                        cmif_precision prec, unsigned flags) {
    if (!out) return CMIF_ERR_INVALID_ARG;
    *out = nullptr;
    cmif_plan p = new (std::nothrow) cmif_plan_s();
    if (!p) return CMIF_ERR_OOM;
    cmif_status st = plan_init(p, H_A, W_A, H_B, W_B, K_A, K_B, prec, flags, D_A, D_B);
    if (st == CMIF_OK) {
        const size_t bytes = plan_bytes(p);
        cudaError_t e = cudaMalloc(&p->mem, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); p->mem = nullptr; st = CMIF_ERR_OOM; }
        else {
            p->mem_bytes = bytes;
            st = plan_carve(p, (char*)p->mem);
        }
    }
    if (st == CMIF_OK) {
        // the forward transforms' second stream (blocking neither way with the legacy stream)
        if (cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st = CMIF_ERR_CUDA;
        }
    }
    if (st == CMIF_OK && (flags & CMIF_FLAG_AUTOTUNE)) st = autotune(p, std::getenv("CMIF_TUNE_CACHE"), nullptr);
    if (st != CMIF_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return CMIF_OK;
}
}  // namespace

cmif_status cmif_plan_create_ex(cmif_plan* out, int H_A, int W_A, int H_B, int W_B, int K_A, int K_B,
                                cmif_precision prec, unsigned flags) {
    return plan_create(out, 1, H_A, W_A, 1, H_B, W_B, K_A, K_B, prec, flags);
}

cmif_status cmif_plan_create_3d(cmif_plan* out, int D_A, int H_A, int W_A, int D_B, int H_B, int W_B, int K_A,
                                int K_B, cmif_precision prec, unsigned flags) {
    return plan_create(out, D_A, H_A, W_A, D_B, H_B, W_B, K_A, K_B, prec, flags);
}

cmif_status cmif_plan_create(cmif_plan* out, int H, int W, int K_A, int K_B, cmif_precision prec) {
    return cmif_plan_create_ex(out, H, W, H, W, K_A, K_B, prec, 0u);
}

cmif_status cmif_plan_destroy(cmif_plan plan) {
    free_plan(plan);
    return CMIF_OK;
}

cmif_status cmif_plan_workspace_bytes(cmif_plan plan, size_t* bytes) {
    if (!plan || !bytes) return CMIF_ERR_INVALID_ARG;
    *bytes = plan->mem_bytes;
    return CMIF_OK;
}

cmif_status cmif_compute(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                         const uint8_t* M_B, double* mi_map, int32_t* n_map, int32_t* counts, double gamma,
                         cmif_peak* peak_dev, void* stream) {
    if (!plan || !A || !B || !mi_map) return CMIF_ERR_INVALID_ARG;
    if (counts && !(plan->flags & CMIF_FLAG_DEBUG_COUNTS)) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    plan->prof.reset();
    int32_t* nm = n_map ? n_map : plan->nbuf;
    std::vector<unsigned char> key;
    key_add(key, 1);
    key_add(key, A); key_add(key, M_A); key_add(key, B); key_add(key, M_B);
    key_add(key, mi_map); key_add(key, nm); key_add(key, counts); key_add(key, gamma); key_add(key, peak_dev);
    Geom g;
    if (!call_geom(plan, gamma, &g)) return CMIF_ERR_INVALID_ARG;
    return run_graph(plan, s, key, [&](cudaStream_t cs) -> cmif_status {
        cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), cs);
        if (e != cudaSuccess) return from_cuda(e);
        if (g.r0 > 0 || g.r1 < g.R) {  // rows outside the window are not computed: zero
            const size_t RC = (size_t)g.R * g.C;
            e = cudaMemsetAsync(mi_map, 0, RC * sizeof(double), cs);
            if (e == cudaSuccess) e = cudaMemsetAsync(nm, 0, RC * sizeof(int32_t), cs);
            if (e == cudaSuccess && counts)
                e = cudaMemsetAsync(counts, 0, RC * sizeof(int32_t) * ((size_t)g.KA * g.KB + g.KA + g.KB), cs);
            if (e != cudaSuccess) return from_cuda(e);
        }
        cmif_status st = compute_map(plan, g, A, M_A, B, M_B, mi_map, nm, counts, cs);
        if (st != CMIF_OK) return st;
        if (peak_dev) {
            plan->prof.begin("peak", cs);
            e = launch_peak(mi_map, nm, g, plan->st, gamma, plan->parts, plan->nparts, 0, peak_dev, cs);
            plan->prof.end(cs);
            if (e != cudaSuccess) return from_cuda(e);
        }
        return CMIF_OK;
    });
}

cmif_status cmif_compute_weighted(cmif_plan plan, const int32_t* A, const double* W_A, const int32_t* B,
                                  const double* W_B, double* mi_map, double* nw_map, double gamma, cmif_peak* peak_dev,
                                  void* stream) {
    if (!plan || !A || !B || !mi_map) return CMIF_ERR_INVALID_ARG;
    if (!(plan->flags & CMIF_FLAG_WEIGHTED) || plan->w64.rows_grid_w <= 0) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    plan->prof.reset();
    Geom g;
    if (!call_geom(plan, gamma, &g)) return CMIF_ERR_INVALID_ARG;
    double* nw = nw_map ? nw_map : plan->w64.args.nw;
    std::vector<unsigned char> key;
    key_add(key, 4);
    key_add(key, A); key_add(key, W_A); key_add(key, B); key_add(key, W_B);
    key_add(key, mi_map); key_add(key, nw); key_add(key, gamma); key_add(key, peak_dev);
    return run_graph(plan, s, key, [&](cudaStream_t cs) -> cmif_status {
        cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(plan->st, 0, sizeof(DevStatus), cs);
        if (e == cudaSuccess && (g.r0 > 0 || g.r1 < g.R)) {  // rows outside the window are not computed: zero
            const size_t RC = (size_t)g.R * g.C;
            e = cudaMemsetAsync(mi_map, 0, RC * sizeof(double), cs);
            if (e == cudaSuccess) e = cudaMemsetAsync(nw, 0, RC * sizeof(double), cs);
        }
        if (e != cudaSuccess) return from_cuda(e);
        PipeArgs<double> a = plan->w64.args;
        a.A = A; a.MA = nullptr; a.B = B; a.MB = nullptr;
        a.WA = W_A; a.WB = W_B; a.weighted = 1;
        a.mi = mi_map; a.nw = nw; a.n = nullptr; a.counts = nullptr; a.st = plan->st;
        a.wait_polls = plan->test_wait_polls;
        a.withhold_row = plan->test_withhold_row;
        a.prof = plan->prof.enabled ? &plan->prof : nullptr;
        a.stages = STAGE_ALL;
        a.prec_slot = 1;
        a.conditional = 0;
        e = run_pipeline<double>(g, a, cs);
        if (e != cudaSuccess) return from_cuda(e);
        e = launch_merge_status(plan->st, plan->st_total, 1, cs);
        if (e == cudaSuccess && peak_dev) {
            plan->prof.begin("peak", cs);
            e = launch_peak_w(mi_map, nw, g, plan->st, gamma, plan->parts, plan->nparts, peak_dev, cs);
            plan->prof.end(cs);
        }
        return from_cuda(e);
    });
}

cmif_status cmif_compute_host(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                              const uint8_t* M_B, double* mi_map, int32_t* n_map, double gamma,
                              cmif_peak* peak_host, void* stream) {
    if (!plan || !A || !B || !mi_map) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    const Geom& g = plan->g;
    const size_t nA = (size_t)g.DA * g.HA * g.WA, nB = (size_t)g.DB * g.HB * g.WB, RC = (size_t)g.R * g.C;
    size_t off = 0;
    const size_t oA = off; off = align_up(off + nA * 4, 256);
    const size_t oB = off; off = align_up(off + nB * 4, 256);
    const size_t oMA = off; off = align_up(off + nA, 256);
    const size_t oMB = off; off = align_up(off + nB, 256);
    const size_t oMI = off; off = align_up(off + RC * 8, 256);
    const size_t oN = off; off = align_up(off + RC * 4, 256);
    const size_t oPk = off; off = align_up(off + sizeof(cmif_peak), 256);
    if (plan->stage_bytes < off) {
        if (plan->stage) cudaFree(plan->stage);
        plan->stage = nullptr;
        plan->stage_bytes = 0;
        if (cudaMalloc(&plan->stage, off) != cudaSuccess) { cudaGetLastError(); return CMIF_ERR_OOM; }
        plan->stage_bytes = off;
    }
    char* b = (char*)plan->stage;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b + oA, A, nA * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + oB, B, nB * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && M_A) e = cudaMemcpyAsync(b + oMA, M_A, nA, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && M_B) e = cudaMemcpyAsync(b + oMB, M_B, nB, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    const bool want_n = n_map || peak_host;
    // Output maps in page-locked host memory are written by the kernels themselves
    // (the device reaches that memory directly: NVLink-C2C on Grace hosts, PCIe
    // elsewhere), as the rows are finished, instead of a copy after the map; other
    // host memory takes a copy from the staging buffer.
    auto direct = [](void* host) -> void* {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, host) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
    };
    double* mi_out = static_cast<double*>(direct(mi_map));
    int32_t* n_out = n_map ? static_cast<int32_t*>(direct(n_map)) : nullptr;
    const bool mi_copy = mi_out == nullptr, n_copy = n_map && n_out == nullptr;
    if (mi_copy) mi_out = (double*)(b + oMI);
    if (!n_out && want_n) n_out = (int32_t*)(b + oN);
    cmif_status st = cmif_compute(plan, (int32_t*)(b + oA), M_A ? (uint8_t*)(b + oMA) : nullptr, (int32_t*)(b + oB),
                                  M_B ? (uint8_t*)(b + oMB) : nullptr, mi_out, want_n ? n_out : nullptr, nullptr,
                                  gamma, peak_host ? (cmif_peak*)(b + oPk) : nullptr, stream);
    if (st != CMIF_OK) return st;
    if (mi_copy) e = cudaMemcpyAsync(mi_map, b + oMI, RC * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && n_copy) e = cudaMemcpyAsync(n_map, b + oN, RC * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && peak_host) e = cudaMemcpyAsync(peak_host, b + oPk, sizeof(cmif_peak), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
}

cmif_status cmif_get_status(cmif_plan plan, cmif_status* device_side, double* max_residual, int* escalations) {
    if (!plan) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    DevStatus h{};
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, plan->st_total, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    if (device_side) {
        *device_side = (h.flags & STATUS_LABEL_RANGE) ? CMIF_ERR_LABEL_RANGE
                     : (h.flags & STATUS_TIMEOUT)     ? CMIF_ERR_TIMEOUT
                     : (h.flags & STATUS_PRECISION)   ? CMIF_ERR_PRECISION
                                                      : CMIF_OK;
    }
    if (max_residual) {
        float f0, f1;
        std::memcpy(&f0, &h.res_bits[0], sizeof(f0));
        std::memcpy(&f1, &h.res_bits[1], sizeof(f1));
        *max_residual = plan->prec == CMIF_AUTO ? std::max(f0, f1) : f0;
    }
    if (escalations) *escalations = h.escalations + h.predicted;
    return CMIF_OK;
}

cmif_status cmif_get_precision_report(cmif_plan plan, int* pairs_predicted, int* pairs_escalated,
                                      double* residual_fp32, double* residual_second) {
    if (!plan) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    DevStatus h{};
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, plan->st_total, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    float f0, f1;
    std::memcpy(&f0, &h.res_bits[0], sizeof(f0));
    std::memcpy(&f1, &h.res_bits[1], sizeof(f1));
    if (pairs_predicted) *pairs_predicted = h.predicted;
    if (pairs_escalated) *pairs_escalated = h.escalations;
    // AUTO keeps the FP32 pairs' and the second-precision pairs' residuals apart;
    // other plans have one authoritative residual
    if (residual_fp32) *residual_fp32 = (plan->prec == CMIF_AUTO || plan->prec == CMIF_FP32) ? (double)f0 : 0.0;
    if (residual_second)
        *residual_second = plan->prec == CMIF_AUTO ? (double)f1 : (plan->prec == CMIF_FP32 ? 0.0 : (double)f0);
    return CMIF_OK;
}

cmif_status cmif_rotate_nn(const int32_t* B, const uint8_t* M_B, int H, int W, double theta, int32_t* B_out,
                           uint8_t* M_out, void* stream) {
    if (!B || !B_out || !M_out || H < 1 || W < 1 || !std::isfinite(theta)) return CMIF_ERR_INVALID_ARG;
    return from_cuda(launch_warp_nn(B, M_B, H, W, theta, B_out, M_out, (cudaStream_t)stream));
}

cmif_status cmif_align_rotations(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                 const uint8_t* M_B, const double* angles_rad_host, int n_angles, double gamma,
                                 int top_k, cmif_peak* topk_dev, double* mi_maps, int32_t* n_maps, void* stream) {
    if (!plan || !A || !B || !angles_rad_host || !topk_dev || plan->g.Dz > 1) return CMIF_ERR_INVALID_ARG;
    if (n_angles < 1 || n_angles > kMaxAngles || top_k < 1 || top_k > n_angles) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    for (int i = 0; i < n_angles; ++i)
        if (!std::isfinite(angles_rad_host[i])) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    plan->prof.reset();
    std::vector<unsigned char> key;
    key_add(key, 2);
    key_add(key, A); key_add(key, M_A); key_add(key, B); key_add(key, M_B);
    key_add(key, gamma); key_add(key, top_k); key_add(key, topk_dev); key_add(key, mi_maps); key_add(key, n_maps);
    key_add(key, n_angles);
    for (int i = 0; i < n_angles; ++i) key_add(key, angles_rad_host[i]);
    return run_graph(plan, s, key, [&](cudaStream_t cs) -> cmif_status {
        return align_core(plan, A, M_A, B, M_B, angles_rad_host, n_angles, gamma, top_k, topk_dev, mi_maps, n_maps,
                          cs);
    });
}

cmif_status cmif_align_two_stage(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                 const uint8_t* M_B, int n_grid, const double* refine_u_host, int n_refine,
                                 double gamma, cmif_peak* best_host, double* best_angle_rad, void* stream) {
    if (!plan || !A || !B || !best_host || !best_angle_rad || plan->g.Dz > 1) return CMIF_ERR_INVALID_ARG;
    if (n_grid < 1 || n_grid > kMaxAngles || n_refine < 0 || n_refine > kMaxAngles || (n_refine > 0 && !refine_u_host))
        return CMIF_ERR_INVALID_ARG;
    for (int i = 0; i < n_refine; ++i)
        if (!(refine_u_host[i] >= 0.0 && refine_u_host[i] <= 1.0)) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    const double two_pi = 6.283185307179586476925286766559;
    PeakRec* slot = reinterpret_cast<PeakRec*>(plan->peaks) + kMaxAngles;  // two records past the per-angle ones
    // (i) grid search over theta_t = 2 pi t / |Omega|
    std::vector<double> grid(n_grid);
    for (int t = 0; t < n_grid; ++t) grid[t] = two_pi * t / n_grid;
    cmif_status st = cmif_align_rotations(plan, A, M_A, B, M_B, grid.data(), n_grid, gamma, 1,
                                          reinterpret_cast<cmif_peak*>(slot), nullptr, nullptr, stream);
    if (st != CMIF_OK) return st;
    PeakRec best{};
    cudaError_t e = cudaMemcpyAsync(&best, slot, sizeof(PeakRec), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    // Alg. 1 keeps the identity (I = 0) unless some transform has I_T > 0
    if (!(best.angle_idx >= 0 && best.mi > 0.0)) best = {-1, 0, 0, 0, 0.0};
    double best_theta = best.angle_idx >= 0 ? grid[best.angle_idx] : 0.0;
    // (ii) random refinement: theta + (2u - 1) 2 pi / |Omega|, continuing Alg. 1's (I, T-hat)
    if (n_refine > 0) {
        std::vector<double> ref(n_refine);
        const double half = two_pi / n_grid;
        for (int i = 0; i < n_refine; ++i) ref[i] = best_theta + (2.0 * refine_u_host[i] - 1.0) * half;
        st = cmif_align_rotations(plan, A, M_A, B, M_B, ref.data(), n_refine, gamma, 1,
                                  reinterpret_cast<cmif_peak*>(slot + 1), nullptr, nullptr, stream);
        if (st != CMIF_OK) return st;
        PeakRec r2{};
        e = cudaMemcpyAsync(&r2, slot + 1, sizeof(PeakRec), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
        if (r2.angle_idx >= 0 && r2.mi > best.mi) {
            best_theta = ref[r2.angle_idx];
            best = r2;
            best.angle_idx += n_grid;
        }
    }
    best_host->angle_idx = best.angle_idx;
    best_host->dy = best.dy;
    best_host->dx = best.dx;
    best_host->n = best.n;
    best_host->mi = best.mi;
    *best_angle_rad = best_theta;
    return CMIF_OK;
}

cmif_status cmif_batch_create(cmif_batch* out, int n_pairs, const cmif_pair_desc* descs, cmif_precision prec,
                              unsigned flags) {
    if (!out) return CMIF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_pairs < 1 || !descs ||
        (flags & ~(CMIF_FLAG_GRAPH | CMIF_FLAG_WINDOW | CMIF_FLAG_NMI | CMIF_FLAG_AUTOTUNE | CMIF_FLAG_BATCH_ANGLES)))
        return CMIF_ERR_INVALID_ARG;
    for (int i = 0; i < n_pairs; ++i) {
        const cmif_pair_desc& d = descs[i];
        if (!d.A || !d.B || d.n_angles < 0 || d.n_angles > kMaxAngles || (d.n_angles > 0 && !d.angles_rad))
            return CMIF_ERR_INVALID_ARG;
        if (!(d.gamma >= 0.0 && d.gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
        for (int k = 0; k < d.n_angles; ++k)
            if (!std::isfinite(d.angles_rad[k])) return CMIF_ERR_INVALID_ARG;
    }
    cmif_batch b = new (std::nothrow) cmif_batch_s();
    if (!b) return CMIF_ERR_OOM;
    auto fail = [&](cmif_status st) {
        for (cmif_plan p : b->plans) { p->mem = nullptr; free_plan(p); }
        if (b->mem) cudaFree(b->mem);
        delete b;
        return st;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(CMIF_ERR_CUDA);
    b->descs.assign(descs, descs + n_pairs);
    size_t max_bytes = 0;
    for (int i = 0; i < n_pairs; ++i) {
        const cmif_pair_desc& d = descs[i];
        b->angles.emplace_back(d.angles_rad, d.angles_rad + d.n_angles);
        cmif_plan p = new (std::nothrow) cmif_plan_s();
        if (!p) return fail(CMIF_ERR_OOM);
        b->plans.push_back(p);
        cmif_status st = plan_init(p, d.H_A, d.W_A, d.H_B, d.W_B, d.K_A, d.K_B, prec,
                                   flags & (CMIF_FLAG_WINDOW | CMIF_FLAG_NMI | CMIF_FLAG_BATCH_ANGLES), 1, 1,
                                   std::max(1, d.n_angles));
        if (st != CMIF_OK) return fail(st);
        max_bytes = std::max(max_bytes, plan_bytes(p));
    }
    // pairs run one after another on one stream, so one workspace serves them all
    const size_t tot_off = align_up(max_bytes, 256);
    if (cudaMalloc(&b->mem, tot_off + 256) != cudaSuccess) { cudaGetLastError(); b->mem = nullptr; return fail(CMIF_ERR_OOM); }
    b->mem_bytes = tot_off + 256;
    for (cmif_plan p : b->plans) {
        cmif_status st = plan_carve(p, (char*)b->mem);
        if (st != CMIF_OK) return fail(st);
    }
    b->total = (DevStatus*)((char*)b->mem + tot_off);
    if (cudaMemset(b->total, 0, sizeof(DevStatus)) != cudaSuccess) return fail(CMIF_ERR_CUDA);
    if (flags & CMIF_FLAG_AUTOTUNE) {  // each size class is timed once (the tuner's cache serves the rest)
        for (cmif_plan p : b->plans) {
            cmif_status st = autotune(p, std::getenv("CMIF_TUNE_CACHE"), nullptr);
            if (st != CMIF_OK) return fail(st);
        }
    }
    b->graph_holder.use_graph = (flags & CMIF_FLAG_GRAPH) != 0;
    b->graph_holder.device = b->device;
    *out = b;
    return CMIF_OK;
}

cmif_status cmif_compute_batch(cmif_batch batch, cmif_peak* results_dev, int32_t* status_dev, void* stream) {
    if (!batch || !results_dev) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(batch->device);
    cudaStream_t s = (cudaStream_t)stream;
    batch->last_stream = s;
    std::vector<unsigned char> key;
    key_add(key, 3);
    key_add(key, results_dev);
    key_add(key, status_dev);
    return run_graph(&batch->graph_holder, s, key, [&](cudaStream_t cs) -> cmif_status {
        cudaError_t e = cudaMemsetAsync(batch->total, 0, sizeof(DevStatus), cs);
        if (e != cudaSuccess) return from_cuda(e);
        for (size_t i = 0; i < batch->plans.size(); ++i) {
            cmif_plan p = batch->plans[i];
            const cmif_pair_desc& d = batch->descs[i];
            cmif_status st;
            if (d.n_angles == 0) {
                e = cudaMemsetAsync(p->st_total, 0, sizeof(DevStatus), cs);
                if (e != cudaSuccess) return from_cuda(e);
                Geom g;
                if (!call_geom(p, d.gamma, &g)) return CMIF_ERR_INVALID_ARG;
                st = compute_map(p, g, d.A, d.M_A, d.B, d.M_B, p->mibuf, p->nbuf, nullptr, cs);
                if (st != CMIF_OK) return st;
                e = launch_peak(p->mibuf, p->nbuf, g, p->st, d.gamma, p->parts, p->nparts, 0, results_dev + i, cs);
                if (e != cudaSuccess) return from_cuda(e);
            } else {
                st = align_core(p, d.A, d.M_A, d.B, d.M_B, batch->angles[i].data(), d.n_angles, d.gamma, 1,
                                results_dev + i, nullptr, nullptr, cs);
                if (st != CMIF_OK) return st;
            }
            if (status_dev) {
                e = launch_status_code(p->st_total, status_dev + i, cs);
                if (e != cudaSuccess) return from_cuda(e);
            }
            e = launch_merge_status(p->st_total, batch->total, p->prec == CMIF_AUTO ? 2 : 0, cs);
            if (e != cudaSuccess) return from_cuda(e);
        }
        return CMIF_OK;
    });
}

cmif_status cmif_batch_get_status(cmif_batch batch, cmif_status* device_side, double* max_residual, int* escalations) {
    if (!batch) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(batch->device);
    DevStatus h{};
    cudaError_t e = cudaStreamSynchronize(batch->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, batch->total, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    if (device_side)
        *device_side = (h.flags & STATUS_LABEL_RANGE) ? CMIF_ERR_LABEL_RANGE
                     : (h.flags & STATUS_TIMEOUT)     ? CMIF_ERR_TIMEOUT
                     : (h.flags & STATUS_PRECISION)   ? CMIF_ERR_PRECISION
                                                      : CMIF_OK;
    if (max_residual) {
        float f0, f1;
        std::memcpy(&f0, &h.res_bits[0], sizeof(f0));
        std::memcpy(&f1, &h.res_bits[1], sizeof(f1));
        *max_residual = std::max(f0, f1);  // res_bits[1] is 0 unless the pairs ran with per-pair precision
    }
    if (escalations) *escalations = h.escalations + h.predicted;
    return CMIF_OK;
}

cmif_status cmif_batch_destroy(cmif_batch batch) {
    if (!batch) return CMIF_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(batch->device);
    cudaDeviceSynchronize();
    for (cmif_plan p : batch->plans) { p->mem = nullptr; free_plan(p); }
    if (batch->mem) cudaFree(batch->mem);
    if (batch->graph_holder.gexec) { cudaGraphExecDestroy(batch->graph_holder.gexec); batch->graph_holder.gexec = nullptr; }
    if (batch->graph_holder.cap_stream) { cudaStreamDestroy(batch->graph_holder.cap_stream); batch->graph_holder.cap_stream = nullptr; }
    if (prev >= 0) cudaSetDevice(prev);
    delete batch;
    return CMIF_OK;
}

cmif_status cmif_plan_set_profiling(cmif_plan plan, int enable) {
    if (!plan) return CMIF_ERR_INVALID_ARG;
    plan->prof.enabled = enable != 0;
    plan->prof.reset();
    return CMIF_OK;
}

cmif_status cmif_plan_stage_times(cmif_plan plan, int max_n, int* n, double* ms, const char** names) {
    if (!plan || !n || max_n < 0) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e != cudaSuccess) return from_cuda(e);
    const int used = (int)plan->prof.used;
    *n = used;
    for (int i = 0; i < used && i < max_n; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, plan->prof.ev[2 * i], plan->prof.ev[2 * i + 1]);
        if (e != cudaSuccess) return from_cuda(e);
        if (ms) ms[i] = t;
        if (names) names[i] = plan->prof.names[i];
    }
    return CMIF_OK;
}

cmif_status cmif_plan_autotune(cmif_plan plan, const char* cache_path, cmif_tuning* out) {
    if (!plan) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e != cudaSuccess) return from_cuda(e);
    return autotune(plan, cache_path, out);
}

cmif_status cmif_plan_set_wait_test(cmif_plan plan, int poll_limit, int withhold_row) {
    if (!plan || poll_limit < 0 || withhold_row < -1) return CMIF_ERR_INVALID_ARG;
    plan->test_wait_polls = poll_limit;
    plan->test_withhold_row = withhold_row;
    return CMIF_OK;
}

cmif_status cmif_entropy_terms(int c0, int n, int64_t* out_dev, void* stream) {
    if (!out_dev || c0 < 0 || n < 0 || (long long)c0 + n > (1LL << 22) + 1) return CMIF_ERR_INVALID_ARG;
    static_assert(sizeof(long long) == sizeof(int64_t), "64-bit terms");
    return from_cuda(launch_entropy_terms(c0, n, reinterpret_cast<long long*>(out_dev), (cudaStream_t)stream));
}

const char* cmif_status_string(cmif_status s) {
    switch (s) {
        case CMIF_OK: return "ok";
        case CMIF_ERR_INVALID_ARG: return "invalid argument";
        case CMIF_ERR_LABEL_RANGE: return "label outside [0, K) under mask";
        case CMIF_ERR_OOM: return "out of device memory";
        case CMIF_ERR_CUDA: return "CUDA error";
        case CMIF_ERR_PRECISION: return "rounding residual above guard in final precision";
        case CMIF_ERR_TIMEOUT: return "device wait timed out";
        case CMIF_ERR_NOT_IMPLEMENTED: return "not implemented";
        case CMIF_ERR_UNSUPPORTED: return "size not supported";
    }
    return "unknown status";
}

}  // extern "C"
