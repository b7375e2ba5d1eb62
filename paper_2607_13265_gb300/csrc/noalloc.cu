// A variant of the filtered primal render that never allocates device memory.
//
// dppt_render_primal keeps the raw (unfiltered) Stokes image of a job seen
// through a camera filter in the context's workspace, which the library grows
// with cudaMalloc when a call needs more than before.  Some callers cannot let
// a library allocate: a process whose device memory is owned by another
// allocator (a framework's caching allocator, a fixed memory budget), a
// latency-critical loop that must not block in the driver's allocator, or
// code that issues work while a stream is being captured.  For them this
// translation unit holds the raw image in a fixed array compiled into the
// library (g_noalloc_raw, 12 MiB: at most 262,144 pixels, e.g. 512 x 512), so
// dppt_render_primal_noalloc only launches kernels and sets memory.
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace dppt {

constexpr long long kNoAllocMaxPixels = 512LL * 512LL;

// Scratch shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) float g_noalloc_raw[kNoAllocMaxPixels * 12];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_raw on the current device (in host code the array's name is
// only a stand-in for it).  Outside stream capture it is resolved again on every call, so
// a context torn down and recreated in between (cudaDeviceReset) cannot leave a stale
// address; a call made while `st` is being captured reuses the address of the device's
// last call outside capture, and fails if there was none.
cudaError_t scratch_address(int device, cudaStream_t st, void** out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_raw);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    } else if (!g_addr[device]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_addr[device];
    return cudaSuccess;
}

cudaError_t launch_bucket(int bucket, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,
                          const LaunchCfg& L, unsigned* status, cudaStream_t st) {
    switch (bucket) {
        case 4: return launch_trace_4(0, S, P, G, T, L, nullptr, status, nullptr, st);
        case 8: return launch_trace_8(0, S, P, G, T, L, nullptr, status, nullptr, st);
        case 16: return launch_trace_16(0, S, P, G, T, L, nullptr, status, nullptr, st);
        case 32: return launch_trace_32(0, S, P, G, T, L, nullptr, status, nullptr, st);
        case 64: return launch_trace_64(0, S, P, G, T, L, nullptr, status, nullptr, st);
        case 128: return launch_trace_128(0, S, P, G, T, L, nullptr, status, nullptr, st);
    }
    return cudaErrorInvalidValue;
}

dppt_status bad(dppt_ctx* ctx, dppt_status code, const std::string& msg) {
    ctx_set_error(ctx, msg.c_str());
    return code;
}

}  // namespace
}  // namespace dppt

using namespace dppt;

extern "C" dppt_status dppt_render_primal_noalloc(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* job,
                                                  const dppt_params* params, float* image, void* stream) {
    if (!ctx) return DPPT_ERR_INVALID_ARG;
    if (!scene || !job || !params || !image) return bad(ctx, DPPT_ERR_INVALID_ARG, "null argument");
    const int device = ctx_device(ctx);
    if (device < 0 || device >= kMaxDevices) return bad(ctx, DPPT_ERR_INVALID_ARG, "device ordinal out of range");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bad(ctx, DPPT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    const dppt_job& j = *job;
    const DScene& S = *scene_view(scene);
    if (j.camera < 0 || j.camera >= scene_num_cameras(scene)) return bad(ctx, DPPT_ERR_INVALID_ARG, "camera index out of range");
    if (j.width < 1 || j.height < 1 || j.spp < 1 || j.spp > (1 << 20) || j.max_depth < 1 || j.max_depth > kMaxDepth)
        return bad(ctx, DPPT_ERR_INVALID_ARG, "bad image size, spp or max_depth");
    if (j.filter < DPPT_FILTER_NONE || j.filter > DPPT_FILTER_QWP_POLARIZER) return bad(ctx, DPPT_ERR_INVALID_ARG, "unknown filter");
    if (j.out_offset < 0 || (j.out_offset & 3) != 0) return bad(ctx, DPPT_ERR_INVALID_ARG, "out_offset must be a non-negative multiple of 4");
    const long long npix = (long long)j.width * j.height;
    if (npix > kNoAllocMaxPixels)
        return bad(ctx, DPPT_ERR_INVALID_ARG, "image of " + std::to_string(npix) + " pixels exceeds the fixed scratch of " +
                                               std::to_string(kNoAllocMaxPixels) + " pixels; use dppt_render_primal");
    const bool filtered = j.filter != DPPT_FILTER_NONE;
    if (filtered && (j.num_angles < 1 || j.num_angles > 512 || j.theta_offset < 0 || !params->theta))
        return bad(ctx, DPPT_ERR_INVALID_ARG, "filtered job needs 1..512 angles and params.theta");
    if ((scene_tex_size(scene) > 0 && !params->tex) || (S.num_ior > 0 && !params->ior) ||
        (S.num_lights > 0 && !params->le) || (S.num_sheets > 0 && !params->sheet))
        return bad(ctx, DPPT_ERR_INVALID_ARG, "params pointer is null");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* base = nullptr;
    if (filtered) {
        e = scratch_address(device, st, &base);
        if (e != cudaSuccess)
            return bad(ctx, DPPT_ERR_CUDA, std::string("scratch address (make one call outside stream capture first): ") +
                                               cudaGetErrorString(e));
    }
    const int block = 128;
    JobTable T;
    std::memset(&T, 0, sizeof T);
    T.njobs = 1;
    DJob& J = T.job[0];
    J.cam = j.camera; J.W = j.width; J.H = j.height; J.spp = j.spp; J.depth = j.max_depth;
    const bool pow2 = (j.spp & (j.spp - 1)) == 0;
    J.red_mode = pow2 && j.spp <= 32 ? 0 : (pow2 ? 1 : 2);
    J.k0 = j.seed ^ ((unsigned long long)(uint32_t)j.pass * 0x9E3779B97F4A7C15ULL);
    J.kn = (j.seed ^ 0x5bd1e995ULL) ^ (3ULL * 0x9E3779B97F4A7C15ULL);
    J.k1 = j.stream;
    J.npaths = npix * j.spp;
    J.chunk_begin = 0;
    J.sig = j.path_sig;
    J.raw = filtered ? static_cast<float*>(base) : image + j.out_offset;
    J.dS = nullptr;
    T.total_chunks = (J.npaths + block - 1) / block;
    if (J.red_mode != 0) {   // the sums accumulate with atomics: start from zero
        e = cudaMemsetAsync(J.raw, 0, (size_t)npix * 12 * sizeof(float), st);
        if (e != cudaSuccess) return bad(ctx, DPPT_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
    }
    int bucket = kMaxDepth;
    for (int b : {4, 8, 16, 32, 64, 128})
        if (j.max_depth <= b) { bucket = b; break; }
    DParams P{params->tex, params->ior, params->le, params->sheet, params->theta};
    DGrads G{nullptr, nullptr, nullptr, nullptr};
    LaunchCfg L{DPPT_SCHED_GRID, block, 0};
    e = launch_bucket(bucket, S, P, G, T, L, ctx_status_word(ctx), st);
    if (e != cudaSuccess) return bad(ctx, DPPT_ERR_CUDA, std::string("primal launch: ") + cudaGetErrorString(e));
    if (filtered) {
        FoldJob f{};
        f.raw = static_cast<const float*>(base);
        f.image = image + j.out_offset;
        f.theta = params->theta + j.theta_offset;
        f.npix = npix;
        f.filter = j.filter;
        f.nang = j.num_angles;
        e = launch_apply_filter(&f, 1, st);
        if (e != cudaSuccess) return bad(ctx, DPPT_ERR_CUDA, std::string("filter launch: ") + cudaGetErrorString(e));
    }
    return DPPT_OK;
}
