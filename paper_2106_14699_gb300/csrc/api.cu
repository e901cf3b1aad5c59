// C ABI of the CMIF library: plans, workspace, launch order, status.
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

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
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr int kMaxAngles = 4096;

int pow2_at_least(int v, int lo) {
    int p = lo;
    while (p < v) p <<= 1;
    return p;
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
    void* small = nullptr;  // st + parts + internal N map in one allocation
    int32_t* nbuf = nullptr;  // N map used when the caller passes no n_map
    double* mibuf = nullptr;  // MI map used by cmif_align_rotations when the caller keeps no maps
    int32_t* wB = nullptr;    // rotated floating image (cmif_align_rotations)
    uint8_t* wM = nullptr;    // its rotated-support mask
    void* peaks = nullptr;    // per-transform peaks, kMaxAngles records
    // host-buffer path staging (allocated lazily by cmif_compute_host)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t last_stream = nullptr;
    Profiler prof;
};

namespace {

cmif_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return CMIF_OK;
    if (e == cudaErrorMemoryAllocation) return CMIF_ERR_OOM;
    return CMIF_ERR_CUDA;
}

template <typename T>
cmif_status alloc_workspace(cmif_plan p, Workspace<T>& w) {
    const Geom& g = p->g;
    const size_t cs = sizeof(cpx<T>);
    const size_t sT1A = (size_t)g.KA * g.HA * g.Qs * cs, sT1B = (size_t)g.KB * g.HB * g.Qs * cs;
    const size_t sFA = (size_t)g.KA * g.Qh * g.P * cs, sFB = (size_t)g.KB * g.Qh * g.P * cs;
    const size_t sY = (size_t)g.KA * g.KB * g.R * g.Qs * cs;
    // Row kernel: the TMEM / TMA variant where it applies (FP32, Q = 1024 or 2048),
    // else B-marginal accumulators in shared memory when they fit, else in global memory.
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
        w.cb_smem = true;
    } else {
        const size_t smem_cb = rows_smem_bytes<T>(g.Q, g.KB, true);
        w.cb_smem = smem_cb <= 200 * 1024;
        e = rows_max_blocks_per_sm<T>(g.Q, g.KB, w.cb_smem, &bps);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (bps < 1) return CMIF_ERR_UNSUPPORTED;
    w.rows_grid = std::min(g.R, bps * p->num_sms);
    const size_t sCB = w.cb_smem ? 0 : (size_t)w.rows_grid * g.KB * g.Q * sizeof(float);
    size_t off = 0;
    const size_t oT1A = off; off = align_up(off + sT1A, 256);
    const size_t oT1B = off; off = align_up(off + sT1B, 256);
    const size_t oFA = off; off = align_up(off + sFA, 256);
    const size_t oFB = off; off = align_up(off + sFB, 256);
    const size_t oY = off; off = align_up(off + sY, 256);
    const size_t oCB = off; off = align_up(off + sCB, 256);
    void* base = nullptr;
    e = cudaMalloc(&base, off);
    if (e != cudaSuccess) { cudaGetLastError(); return CMIF_ERR_OOM; }
    w.base = base;
    w.bytes = off;
    char* b = (char*)base;
    w.args.T1A = (cpx<T>*)(b + oT1A);
    w.args.T1B = (cpx<T>*)(b + oT1B);
    w.args.FA = (cpx<T>*)(b + oFA);
    w.args.FB = (cpx<T>*)(b + oFB);
    w.args.Y = (cpx<T>*)(b + oY);
    w.args.cb_global = w.cb_smem ? nullptr : (float*)(b + oCB);
    w.args.rows_grid = w.rows_grid;
    w.args.cb_smem = w.cb_smem;
    return CMIF_OK;
}

void free_plan(cmif_plan p) {
    if (!p) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    if (p->w32.base) cudaFree(p->w32.base);
    if (p->w64.base) cudaFree(p->w64.base);
    if (p->ws32.base) cudaFree(p->ws32.base);
    if (p->small) cudaFree(p->small);
    if (p->stage) cudaFree(p->stage);
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
             int32_t* n, int32_t* counts, DevStatus* st) {
    a.A = A;
    a.MA = MA;
    a.B = B;
    a.MB = MB;
    a.mi = mi;
    a.n = n;
    a.counts = counts;
    a.st = st;
}

// One full map into (mi, n, counts); its status in p->st (reset here) is folded
// into p->st_total.  stages32 selects the FP32 stages (A's transforms may be
// reused across calls); an FP64 pass always recomputes everything.
cmif_status compute_map(cmif_plan p, const int32_t* A, const uint8_t* MA, const int32_t* B, const uint8_t* MB,
                        double* mi, int32_t* n, int32_t* counts, cudaStream_t s, unsigned stages32 = STAGE_ALL) {
    const Geom& g = p->g;
    cudaError_t e0 = cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s);
    if (e0 != cudaSuccess) return from_cuda(e0);
    if (p->prec == CMIF_FP32 || p->prec == CMIF_AUTO) {
        PipeArgs<float> a = p->w32.args;
        fill_io(a, A, MA, B, MB, mi, n, counts, p->st);
        a.prof = p->prof.enabled ? &p->prof : nullptr;
        a.stages = stages32;
        a.prec_slot = 0;
        a.conditional = 0;
        cudaError_t e = run_pipeline<float>(g, a, s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (p->prec == CMIF_AUTO) {
        cudaError_t e = launch_check_escalate(p->st, s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    // second tier: the plan's FP64 / split precision, or AUTO's re-run (gated on the device)
    const cmif_precision second = (p->prec == CMIF_AUTO) ? p->tier2 : p->prec;
    if (p->prec != CMIF_FP32) {
        const int cond = (p->prec == CMIF_AUTO) ? 1 : 0;
        cudaError_t e;
        if (second == CMIF_FP64) {
            PipeArgs<double> a = p->w64.args;
            fill_io(a, A, MA, B, MB, mi, n, counts, p->st);
            a.prof = p->prof.enabled ? &p->prof : nullptr;
            a.stages = STAGE_ALL;
            a.prec_slot = 1;
            a.conditional = cond;
            e = run_pipeline<double>(g, a, s);
        } else {
            PipeArgs<df32> a = p->ws32.args;
            fill_io(a, A, MA, B, MB, mi, n, counts, p->st);
            a.prof = p->prof.enabled ? &p->prof : nullptr;
            a.stages = STAGE_ALL;
            a.prec_slot = 1;
            a.conditional = cond;
            e = run_pipeline<df32>(g, a, s);
        }
        if (e != cudaSuccess) return from_cuda(e);
    }
    const int slot_default = (p->prec == CMIF_FP64 || p->prec == CMIF_SPLIT32) ? 1 : 0;
    p->prof.begin("finalize", s);
    cudaError_t e = launch_finalize(p->st, 1, slot_default, s);
    if (e == cudaSuccess) e = launch_merge_status(p->st, p->st_total, slot_default, s);
    p->prof.end(s);
    return from_cuda(e);
}

}  // namespace

extern "C" {

cmif_status cmif_plan_create_ex(cmif_plan* out, int H_A, int W_A, int H_B, int W_B, int K_A, int K_B,
                                cmif_precision prec, unsigned flags) {
    if (!out) return CMIF_ERR_INVALID_ARG;
    *out = nullptr;
    if (H_A < 1 || W_A < 1 || H_B < 1 || W_B < 1 || K_A < 1 || K_B < 1 || K_A > 64 || K_B > 64)
        return CMIF_ERR_INVALID_ARG;
    if ((long long)H_A * W_A > (1LL << 22) || (long long)H_B * W_B > (1LL << 22)) return CMIF_ERR_INVALID_ARG;
    if (flags & ~CMIF_FLAG_DEBUG_COUNTS) return CMIF_ERR_INVALID_ARG;
    if (prec != CMIF_FP32 && prec != CMIF_SPLIT32 && prec != CMIF_FP64 && prec != CMIF_AUTO) return CMIF_ERR_INVALID_ARG;
    Geom g{};
    g.HA = H_A; g.WA = W_A; g.HB = H_B; g.WB = W_B; g.KA = K_A; g.KB = K_B;
    g.R = H_A + H_B - 1;
    g.C = W_A + W_B - 1;
    g.P = pow2_at_least(g.R, 16);
    g.Q = pow2_at_least(g.C, 16);
    if (g.P > 4096 || g.Q > 4096) return CMIF_ERR_UNSUPPORTED;
    g.Qh = g.Q / 2 + 1;
    g.Qs = (int)align_up((size_t)g.Qh, 4);

    cmif_plan p = new (std::nothrow) cmif_plan_s();
    if (!p) return CMIF_ERR_OOM;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return CMIF_ERR_CUDA; }
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { delete p; return CMIF_ERR_CUDA; }
    p->g = g;
    p->prec = prec;
    p->flags = flags;
    cmif_status st = CMIF_OK;
    if (prec == CMIF_FP32 || prec == CMIF_AUTO) {
        st = alloc_workspace<float>(p, p->w32);
        p->has32 = (st == CMIF_OK);
    }
    const char* t2 = std::getenv("CMIF_AUTO_TIER2");  // "fp64" makes AUTO re-run in FP64 instead of split FP32
    p->tier2 = (t2 && std::strcmp(t2, "fp64") == 0) ? CMIF_FP64 : CMIF_SPLIT32;
    if (st == CMIF_OK && (prec == CMIF_FP64 || (prec == CMIF_AUTO && p->tier2 == CMIF_FP64))) {
        st = alloc_workspace<double>(p, p->w64);
        p->has64 = (st == CMIF_OK);
    }
    if (st == CMIF_OK && (prec == CMIF_SPLIT32 || (prec == CMIF_AUTO && p->tier2 == CMIF_SPLIT32))) {
        st = alloc_workspace<df32>(p, p->ws32);
    }
    if (st == CMIF_OK) {
        Tw<float> tf;
        Tw<double> td;
        Tw<df32> ts;
        e = get_twiddles(p->device, &tf, &td, &ts);
        if (e != cudaSuccess) st = from_cuda(e);
        p->w32.args.tw = tf;
        p->w64.args.tw = td;
        p->ws32.args.tw = ts;
    }
    if (st == CMIF_OK) {
        p->nparts = 2 * p->num_sms;
        const size_t o_tot = align_up(sizeof(DevStatus), 256);
        const size_t o_parts = o_tot + align_up(sizeof(DevStatus), 256);
        const size_t o_n = align_up(o_parts + (size_t)p->nparts * sizeof(PeakPart), 256);
        const size_t o_mi = align_up(o_n + (size_t)g.R * g.C * sizeof(int32_t), 256);
        const size_t o_wB = align_up(o_mi + (size_t)g.R * g.C * sizeof(double), 256);
        const size_t o_wM = align_up(o_wB + (size_t)g.HB * g.WB * sizeof(int32_t), 256);
        const size_t o_pk = align_up(o_wM + (size_t)g.HB * g.WB, 256);
        const size_t bytes = o_pk + (size_t)kMaxAngles * sizeof(PeakRec);
        e = cudaMalloc(&p->small, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); st = CMIF_ERR_OOM; }
        else {
            char* sb = (char*)p->small;
            p->st = (DevStatus*)sb;
            p->st_total = (DevStatus*)(sb + o_tot);
            p->parts = (PeakPart*)(sb + o_parts);
            p->nbuf = (int32_t*)(sb + o_n);
            p->mibuf = (double*)(sb + o_mi);
            p->wB = (int32_t*)(sb + o_wB);
            p->wM = (uint8_t*)(sb + o_wM);
            p->peaks = sb + o_pk;
            if (cudaMemset(p->st_total, 0, sizeof(DevStatus)) != cudaSuccess) st = CMIF_ERR_CUDA;
            if (cudaMemset(p->st, 0, sizeof(DevStatus)) != cudaSuccess) st = CMIF_ERR_CUDA;
        }
    }
    if (st != CMIF_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return CMIF_OK;
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
    *bytes = plan->w32.bytes + plan->w64.bytes + plan->ws32.bytes;
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
    cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return from_cuda(e);
    int32_t* nm = n_map ? n_map : plan->nbuf;
    cmif_status st = compute_map(plan, A, M_A, B, M_B, mi_map, nm, counts, s);
    if (st != CMIF_OK) return st;
    if (peak_dev) {
        const Geom& g = plan->g;
        plan->prof.begin("peak", s);
        e = launch_peak(mi_map, nm, (long long)g.R * g.C, plan->st, gamma, plan->parts, plan->nparts, g.HA, g.WA,
                        g.C, 0, peak_dev, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return CMIF_OK;
}

cmif_status cmif_compute_host(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                              const uint8_t* M_B, double* mi_map, int32_t* n_map, double gamma,
                              cmif_peak* peak_host, void* stream) {
    if (!plan || !A || !B || !mi_map) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    const Geom& g = plan->g;
    const size_t nA = (size_t)g.HA * g.WA, nB = (size_t)g.HB * g.WB, RC = (size_t)g.R * g.C;
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
    cmif_status st = cmif_compute(plan, (int32_t*)(b + oA), M_A ? (uint8_t*)(b + oMA) : nullptr, (int32_t*)(b + oB),
                                  M_B ? (uint8_t*)(b + oMB) : nullptr, (double*)(b + oMI),
                                  want_n ? (int32_t*)(b + oN) : nullptr, nullptr, gamma,
                                  peak_host ? (cmif_peak*)(b + oPk) : nullptr, stream);
    if (st != CMIF_OK) return st;
    e = cudaMemcpyAsync(mi_map, b + oMI, RC * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && n_map) e = cudaMemcpyAsync(n_map, b + oN, RC * 4, cudaMemcpyDeviceToHost, s);
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
                     : (h.flags & STATUS_PRECISION)   ? CMIF_ERR_PRECISION
                     : (h.flags & STATUS_TIMEOUT)     ? CMIF_ERR_TIMEOUT
                                                      : CMIF_OK;
    }
    if (max_residual) {
        float f;
        std::memcpy(&f, &h.res_bits[0], sizeof(f));
        *max_residual = f;
    }
    if (escalations) *escalations = h.escalations;
    return CMIF_OK;
}

cmif_status cmif_rotate_nn(const int32_t* B, const uint8_t* M_B, int H, int W, double theta, int32_t* B_out,
                           uint8_t* M_out, void* stream) {
    if (!B || !B_out || !M_out || H < 1 || W < 1 || !std::isfinite(theta)) return CMIF_ERR_INVALID_ARG;
    return from_cuda(launch_warp_nn(B, M_B, H, W, theta, B_out, M_out, (cudaStream_t)stream));
}

cmif_status cmif_align_rotations(cmif_plan plan, const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                 const uint8_t* M_B, const double* angles_rad_host, int n_angles, double gamma,
                                 int top_k, cmif_peak* topk_dev, double* mi_maps, void* stream) {
    if (!plan || !A || !B || !angles_rad_host || !topk_dev) return CMIF_ERR_INVALID_ARG;
    if (n_angles < 1 || n_angles > kMaxAngles || top_k < 1 || top_k > n_angles) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    for (int i = 0; i < n_angles; ++i)
        if (!std::isfinite(angles_rad_host[i])) return CMIF_ERR_INVALID_ARG;
    DeviceGuard dg(plan->device);
    const Geom& g = plan->g;
    const size_t RC = (size_t)g.R * g.C;
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    plan->prof.reset();
    cudaError_t e = cudaMemsetAsync(plan->st_total, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) return from_cuda(e);
    PeakRec* peaks = reinterpret_cast<PeakRec*>(plan->peaks);
    for (int i = 0; i < n_angles; ++i) {
        plan->prof.begin("warp_nn", s);
        e = launch_warp_nn(B, M_B, g.HB, g.WB, angles_rad_host[i], plan->wB, plan->wM, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
        double* mi = mi_maps ? mi_maps + (size_t)i * RC : plan->mibuf;
        const unsigned stages = (i == 0) ? STAGE_ALL : (STAGE_FWD_B | STAGE_PAIRS);
        cmif_status cs = compute_map(plan, A, M_A, plan->wB, plan->wM, mi, plan->nbuf, nullptr, s, stages);
        if (cs != CMIF_OK) return cs;
        plan->prof.begin("peak", s);
        e = launch_peak(mi, plan->nbuf, (long long)RC, plan->st, gamma, plan->parts, plan->nparts, g.HA, g.WA, g.C,
                        i, peaks + i, s);
        plan->prof.end(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    plan->prof.begin("topk", s);
    e = launch_topk(peaks, n_angles, top_k, topk_dev, s);
    plan->prof.end(s);
    return from_cuda(e);
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
