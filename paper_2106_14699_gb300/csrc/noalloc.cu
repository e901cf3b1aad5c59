// cmif_compute_noalloc: the CMIF map for callers that may not allocate device
// memory.  The paper has no counterpart; this is a deployment convenience.
//
// All scratch (FP32 twiddle tables, status word, peak partials, N map, and the
// transform workspace) lives in one file-scope device array of fixed size.
// Its device address is obtained once per device with cudaGetSymbolAddress:
// in host code the array's name is only a host-side stand-in and must never
// be handed to a kernel.
#include <cstring>
#include <mutex>
#include <vector>

#include "cmif.h"
#include "kernels.cuh"
#include "misc.h"
#include "pipeline.cuh"

namespace cmif {
namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;  // the whole scratch: 64 MiB per GPU, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct NoAllocDevice {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    Tw<float> tw{};
    size_t tw_bytes = 0;
    int num_sms = 0;
};

std::mutex g_mu;
NoAllocDevice g_dev[64];

bool is_set_up(int device) {
    std::lock_guard<std::mutex> lk(g_mu);
    return device >= 0 && device < 64 && g_dev[device].base != nullptr;
}

// One-time set-up on the current device: resolve the array's device address and
// upload the twiddle tables into its head (a synchronous copy, no allocation).
cudaError_t setup(int device, NoAllocDevice** out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    NoAllocDevice& d = g_dev[device];
    if (!d.base) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        std::vector<float> host;
        size_t off_n[14], off_sq[6], off_n3[12];
        twiddle_table_f32(host, off_n, off_sq, off_n3);
        const size_t bytes = host.size() * sizeof(float);
        e = cudaMemcpy(ptr, host.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        const cpx<float>* t = reinterpret_cast<const cpx<float>*>(ptr);
        for (int l = 0; l < 14; ++l) d.tw.n[l] = t + off_n[l];
        for (int l = 0; l < 6; ++l) d.tw.sq[l] = t + off_sq[l];
        for (int l = 0; l < 12; ++l) d.tw.n3[l] = t + off_n3[l];
        d.tw_bytes = up256(bytes);
        d.base = reinterpret_cast<unsigned char*>(ptr);
    }
    *out = &d;
    return cudaSuccess;
}

// Device-side status of the map as a cmif_status code.
__global__ void k_status_code(const DevStatus* st, int32_t* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const unsigned f = st->flags;
        *out = (f & STATUS_LABEL_RANGE) ? CMIF_ERR_LABEL_RANGE
             : (f & STATUS_TIMEOUT)     ? CMIF_ERR_TIMEOUT
             : (f & STATUS_PRECISION)   ? CMIF_ERR_PRECISION
                                        : CMIF_OK;
    }
}

cmif_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return CMIF_OK;
    return CMIF_ERR_CUDA;
}

}  // namespace
}  // namespace cmif

using namespace cmif;

extern "C" cmif_status cmif_compute_noalloc(int H_A, int W_A, int H_B, int W_B, int K_A, int K_B,
                                            const int32_t* A, const uint8_t* M_A, const int32_t* B,
                                            const uint8_t* M_B, double* mi_map, int32_t* n_map, double gamma,
                                            cmif_peak* peak_dev, int32_t* status_dev, void* stream) {
    if (!A || !B || !mi_map) return CMIF_ERR_INVALID_ARG;
    if (H_A < 1 || W_A < 1 || H_B < 1 || W_B < 1 || K_A < 1 || K_B < 1 || K_A > 64 || K_B > 64)
        return CMIF_ERR_INVALID_ARG;
    if ((long long)H_A * W_A > (1LL << 22) || (long long)H_B * W_B > (1LL << 22)) return CMIF_ERR_INVALID_ARG;
    if (!(gamma >= 0.0 && gamma <= 1.0)) return CMIF_ERR_INVALID_ARG;
    Geom g{};
    g.HA = H_A; g.WA = W_A; g.HB = H_B; g.WB = W_B; g.KA = K_A; g.KB = K_B;
    g.R = H_A + H_B - 1;
    g.C = W_A + W_B - 1;
    g.r0 = 0; g.r1 = g.R; g.c0 = 0; g.c1 = g.C;  // the whole map
    g.DA = 1; g.DB = 1; g.Dz = 1; g.R2 = g.R; g.units = 1;  // images, one map
    g.P = 16;
    while (g.P < g.R) g.P <<= 1;
    g.Q = 16;
    while (g.Q < g.C) g.Q <<= 1;
    if (g.P > 4096 || g.Q > 4096) return CMIF_ERR_UNSUPPORTED;
    g.Qh = g.Q / 2 + 1;
    g.Qs = (g.Qh + 3) / 4 * 4;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return CMIF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (!is_set_up(device)) {
        // The first call on a device uploads the twiddle tables with a synchronous
        // copy, which a stream capture in progress would invalidate: refuse it.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return CMIF_ERR_CUDA;
        if (cap != cudaStreamCaptureStatusNone) return CMIF_ERR_INVALID_ARG;
    }
    NoAllocDevice* d = nullptr;
    cudaError_t e = setup(device, &d);
    if (e != cudaSuccess) return to_status(e);

    // The B-marginals must fit in shared memory (no global scratch slice here).
    const size_t smem = rows_smem_bytes<float>(g.Q, g.KB, true);
    if (smem > 200 * 1024) return CMIF_ERR_UNSUPPORTED;
    int bps = 0;
    e = rows_max_blocks_per_sm<float>(g.Q, g.KB, true, &bps);
    if (e != cudaSuccess) return to_status(e);
    if (bps < 1) return CMIF_ERR_UNSUPPORTED;

    // Carve the fixed array: [twiddles | status | peak partials | N map | T1A | T1B | FA | FB | Y | counter].
    const size_t cs = sizeof(cpx<float>);
    const int nparts = 2 * d->num_sms;
    size_t off = d->tw_bytes;
    const size_t oSt = off; off = up256(off + sizeof(DevStatus));
    const size_t oParts = off; off = up256(off + (size_t)nparts * sizeof(PeakPart));
    const size_t oN = off; off = up256(off + (n_map ? 0 : (size_t)g.R * g.C * sizeof(int32_t)));
    const size_t oT1A = off; off = up256(off + (size_t)g.KA * g.HA * g.Qs * cs);
    const size_t oT1B = off; off = up256(off + (size_t)g.KB * g.HB * g.Qs * cs);
    const size_t oFA = off; off = up256(off + (size_t)g.KA * g.Qh * g.P * cs);
    const size_t oFB = off; off = up256(off + (size_t)g.KB * g.Qh * g.P * cs);
    const size_t oY = off; off = up256(off + (size_t)g.KA * g.KB * g.R * g.Qs * cs);
    const size_t oCtr = off; off = up256(off + sizeof(int));
    if (off > kNoAllocBytes) return CMIF_ERR_UNSUPPORTED;

    unsigned char* b = d->base;
    DevStatus* st = reinterpret_cast<DevStatus*>(b + oSt);
    e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);  // the status word must start at zero every call
    if (e != cudaSuccess) return to_status(e);
    int32_t* nm = n_map ? n_map : reinterpret_cast<int32_t*>(b + oN);

    PipeArgs<float> a{};
    a.A = A; a.MA = M_A; a.B = B; a.MB = M_B;
    a.T1A = reinterpret_cast<cpx<float>*>(b + oT1A);
    a.T1B = reinterpret_cast<cpx<float>*>(b + oT1B);
    a.FA = reinterpret_cast<cpx<float>*>(b + oFA);
    a.FB = reinterpret_cast<cpx<float>*>(b + oFB);
    a.Y = reinterpret_cast<cpx<float>*>(b + oY);
    a.cb_global = nullptr;
    a.work_ctr = reinterpret_cast<int*>(b + oCtr);
    a.tw = d->tw;
    a.mi = mi_map; a.n = nm; a.counts = nullptr; a.st = st;
    a.prec_slot = 0; a.conditional = 0;
    a.rows_grid = std::min(g.R, bps * d->num_sms);
    a.num_sms = d->num_sms;
    a.cb_smem = true;
    a.prof = nullptr;
    a.tm_cols = 0;
    a.wait_polls = 0;
    a.withhold_row = -1;
    e = run_pipeline<float>(g, a, s);
    if (e != cudaSuccess) return to_status(e);
    e = launch_finalize(st, 0, 0, s);
    if (e != cudaSuccess) return to_status(e);
    if (peak_dev) {
        e = launch_peak(mi_map, nm, g, st, gamma, reinterpret_cast<PeakPart*>(b + oParts), nparts, 0, peak_dev, s);
        if (e != cudaSuccess) return to_status(e);
    }
    if (status_dev) {
        k_status_code<<<1, 32, 0, s>>>(st, status_dev);
        e = cudaGetLastError();
        if (e != cudaSuccess) return to_status(e);
    }
    return CMIF_OK;
}
