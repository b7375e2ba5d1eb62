// Structures shared by the host side of the library and its kernels.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "dppt.h"

namespace dppt {

constexpr int kMaxJobsPerLaunch = 64;
constexpr int kBvhStack = 64;
constexpr int kMaxDepth = 128;      // surface vertices per path (largest cache bucket)
// traversal of the 4-wide BVH (1) or of the binary one (0)
#ifndef DPPT_BVH4
#define DPPT_BVH4 1
#endif

struct DMat {
    int type, albedo_tex, rough_tex, ior_index, sheet_index, normal_tex;
    float eta_re, eta_im, t1[3], t2[3], retard, emission;
};
struct DLight { float o[3], e1[3], e2[3], n[3], area; };
struct DTex { long long off; int w, h, ch, pad; };
struct DCam { float org[3], fwd[3], right[3], up[3], tanh; };

// BVH: two-wide nodes holding the boxes of both children (4 x float4 = 64 B):
//   n0 = (lx0, lx1, ly0, ly1), n1 = (rx0, rx1, ry0, ry1), n2 = (lz0, lz1, rz0, rz1),
//   n3 = (left ref, right ref, -, -) as ints.  A ref >= 0 is an inner node; a
//   ref < 0 is a leaf ~(first | count << 25) over the BVH-ordered triangles.
// Triangles (3 x float4 = 48 B, BVH order): (v0, original id), (e1, 0), (e2, 0).
struct DScene {
    const float4* nodes;    // binary BVH: 4 float4 per node
    const float4* nodes4;   // the same tree collapsed to 4 children per node: 8 float4 per node
    const float4* tris;
    int num_tris;
    int num_nodes;
    const int* tri_mat;     // original triangle order
    const int* tri_light;
    const float* tri_uv;    // [F][6]
    const float* tri_tan;   // [F][3] dP/du per triangle (original order), or null without normal maps
    const float4* spheres;
    const int* sph_mat;
    int num_spheres;
    int num_lights;
    const DMat* mats;
    const DLight* lights;
    const DTex* tex;
    const DCam* cams;
    float eps;
    int num_ior, num_sheets;
    int scatter_lane;       // adjoint: texel gradients one atomic per lane (1) or per warp group (0)
    int sgrad_lanes;        // adjoint: scalar-gradient accumulators with a copy per lane (1) or one (0)
    int tex_shared;         // adjoint: texel gradients summed in the block's accumulators too (the
                            // texel floats, when every texture together is that small), or 0
    int mat_types;          // bit t set when a triangle or sphere uses a material of type t
};

// Scalar gradients (indices of refraction, sheet angles, emitter Stokes vectors) are summed
// per block in shared memory and flushed with one global atomic per block and scalar.  With
// sgrad_lanes (the wavefront replay) each scalar has 32 copies when they fit in 16 KB: lane
// l of a warp adds to copy l, so the lanes of a warp adding to one scalar use 32 banks
// instead of serialising on one address.  The megakernels keep one copy: their thread-local
// caches live in L1, which a larger shared-memory carveout would shrink.  When a scene's
// textures hold few texels in all (tex_shared), their gradients join the accumulators after
// the scalars: every replayed vertex adds to the same few texels, and global atomics on them
// serialise across the whole GPU.
inline __host__ __device__ int sgrad_texel_base(const DScene& S) { return S.num_ior + S.num_sheets + 12 * S.num_lights; }
inline __host__ __device__ int sgrad_scalars(const DScene& S) { return sgrad_texel_base(S) + S.tex_shared; }
// the largest accumulator count that keeps 32 copies within 16 KB
constexpr int kSharedGradFloats = 16384 / (32 * 4);
inline __host__ __device__ int sgrad_copies(const DScene& S) {
    return S.sgrad_lanes && sgrad_scalars(S) * 32 * (int)sizeof(float) <= 16384 ? 32 : 1;
}
inline __host__ __device__ size_t sgrad_bytes(const DScene& S) {
    return sizeof(float) * (size_t)sgrad_scalars(S) * (size_t)sgrad_copies(S);
}

struct DParams {
    const float* tex;
    const float* ior;
    const float* le;
    const float* sheet;
    const float* theta;
};
struct DGrads {
    float* tex;
    float* ior;
    float* le;
    float* sheet;
};

// One render job as the kernels see it.  A launch numbers the blocks' chunks
// of paths consecutively over its jobs (chunk_begin); a chunk never straddles
// two jobs.  red_mode selects how a pixel's paths are summed (see pixel_reduce).
struct DJob {
    int cam, W, H, spp, depth, red_mode;
    unsigned long long k0, k1;
    unsigned long long kn;   // key of the basic polarized PRB's noise stream (seed ^ 0x5bd1e995, pass 3)
    long long npaths;
    long long chunk_begin;
    float* raw;            // mean raw sensor-frame Stokes per pixel [H*W][12] (primal: image or
                           // workspace; adjoint: S_adj for the filter-angle gradients, or null)
    const float* dS;       // adjoint: per-pixel adjoint of the raw image [H*W][12]
    unsigned* sig;         // optional per-path signature
};
struct JobTable {
    DJob job[kMaxJobsPerLaunch];
    int njobs;
    int pad;
    long long total_chunks;
};

struct LaunchCfg {
    int schedule, block, grid;
};

// Kernel launches per stage, and (when timing is on) CUDA events recorded on
// the launching stream around every record: one launch, or several (begin's `kernels`)
// issued back to back for one stage.
enum Stage {
    kStagePrimal = 0, kStageAdjoint, kStageWfInit, kStageWfExtend, kStageWfShade, kStageWfShadow,
    kStageWfCache, kStageWfReplay, kStageWfSweep, kStageWfPixels, kStageFilter, kStageCount
};
struct StageLog {
    int64_t launches[kStageCount] = {0};
    double ms[kStageCount] = {0};
    bool timing = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> spare;
    cudaEvent_t take() {
        if (spare.empty()) { cudaEvent_t e = nullptr; cudaEventCreate(&e); return e; }
        cudaEvent_t e = spare.back(); spare.pop_back(); return e;
    }
    int begin(int stage, cudaStream_t st, int kernels = 1) {
        launches[stage] += kernels;
        if (!timing) return -1;
        Rec r{stage, take(), take()};
        cudaEventRecord(r.a, st);
        recs.push_back(r);
        return (int)recs.size() - 1;
    }
    void end(int tok, cudaStream_t st) {
        if (tok >= 0) cudaEventRecord(recs[tok].b, st);
    }
    void collect() {
        for (Rec& r : recs) {
            cudaEventSynchronize(r.b);
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
            else cudaGetLastError();   // a failed query must not surface as the next launch's error
            spare.push_back(r.a);
            spare.push_back(r.b);
        }
        recs.clear();
    }
    ~StageLog() {
        for (Rec& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (cudaEvent_t e : spare) cudaEventDestroy(e);
    }
};

// megakernel entry points, one set per cache-depth bucket (trace_d<B>.cu);
// mode 0 primal, 1 adjoint, 2 instrumented primal (work counts, no image)
#define DPPT_DECLARE_BUCKET(B)                                                                                   \
    cudaError_t launch_trace_##B(int mode, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, \
                                 const LaunchCfg& L, unsigned long long* counter, unsigned* status,             \
                                 unsigned long long* work, cudaStream_t st);                                    \
    cudaError_t trace_attributes_##B(int mode, cudaFuncAttributes* a);                                         \
    int trace_occupancy_##B(int mode, int block, size_t smem);                                                  \
    /* the sweep schedule's forward-sweep kernel of the bucket (wavefront.cuh) */                               \
    cudaError_t sweep_attributes_##B(cudaFuncAttributes* a);                                                    \
    int sweep_occupancy_##B(int block);
DPPT_DECLARE_BUCKET(4)
DPPT_DECLARE_BUCKET(8)
DPPT_DECLARE_BUCKET(16)
DPPT_DECLARE_BUCKET(32)
DPPT_DECLARE_BUCKET(64)
DPPT_DECLARE_BUCKET(128)
#undef DPPT_DECLARE_BUCKET

// hybrid cached replay (hybrid_k<K>.cu): adjoint megakernels with checkpoint interval K
// for depth buckets 8..128
struct HybridCfg { float gamma, eps; };
#define DPPT_DECLARE_HYBRID(K)                                                                                     \
    cudaError_t launch_hybrid_##K(int bucket, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, \
                                  const LaunchCfg& L, unsigned long long* counter, unsigned* status, HybridCfg hc, \
                                  cudaStream_t st);                                                               \
    cudaError_t hybrid_attributes_##K(int bucket, cudaFuncAttributes* a);                                         \
    int hybrid_occupancy_##K(int bucket, int block, size_t smem);
// basic polarized PRB (pprb.cu): the cache-free adjoint megakernel of Sec. 4.1-4.2
cudaError_t launch_pprb(const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, const LaunchCfg& L,
                        unsigned long long* counter, unsigned* status, float sigma, cudaStream_t st);
cudaError_t pprb_attributes(cudaFuncAttributes* a);
int pprb_occupancy(int block, size_t smem);
DPPT_DECLARE_HYBRID(4)
DPPT_DECLARE_HYBRID(8)
DPPT_DECLARE_HYBRID(16)
#undef DPPT_DECLARE_HYBRID

// wavefront schedule (wavefront.cu): workspace bytes for waves of Q paths with a cache of
// `cap` vertices (k > 1: the hybrid replay's checkpoints every k vertices instead of the
// per-vertex cache), and the run of every job of a table (several jobs share a wave).
// sweep > 0 (the adjoint of schedule DPPT_SCHED_SWEEP, fully cached replay): each wave's
// forward sweep runs in the megakernel of cache-depth bucket `sweep` instead of the stage
// kernels.
struct WfHybrid { int k; float gamma, eps; };   // k = 1: the fully cached replay
// A second stream of the context with two events: a replay iteration runs its small bins on
// it beside the diffuse bin (forked from and joined back into the launching stream, so the
// launches stay one capturable sequence on that stream)
struct SideStream { cudaStream_t st; cudaEvent_t fork, join; };
size_t wavefront_bytes(long long Q, int cap, int k);
cudaError_t run_wavefront(int mode, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,
                          void* ws, long long Q, int cap, int block, const WfHybrid& hy, int sweep, unsigned* status,
                          cudaStream_t st, const SideStream* side, StageLog* log);

// read-only views of the opaque context and scene (host.cpp), for entry points
// implemented in other translation units
int ctx_device(const dppt_ctx* c);
unsigned* ctx_status_word(const dppt_ctx* c);
void ctx_set_error(dppt_ctx* c, const char* msg);
const DScene* scene_view(const dppt_scene* s);
int scene_num_cameras(const dppt_scene* s);
int64_t scene_tex_size(const dppt_scene* s);

// Camera-filter folds, every job of a call in one launch (one per kMaxFoldJobs jobs;
// fold_launches counts them).  A job's fields by fold:
//   apply_filter:          image[a][pix] = C(theta_a) raw[pix]
//   filter_adjoint_input:  dS[pix] = sum_a C_a^T dimage_a[pix]
//   theta_grad:            dtheta_a += sum_pix dimage_a[pix]^T dC_a/dtheta S_adj[pix]
//   l2_loss:               *loss += scale sum_a sum_pix |C_a raw - target_a|^2
//   l2_adjoint_input:      dS[pix] = 2 scale sum_a C_a^T (C_a raw - target_a)
//   l2_theta_grad:         dtheta_a += 2 scale sum_pix (C_a raw - target_a)^T dC_a S_adj[pix]
// The L2 folds take a job without a camera filter as filter DPPT_FILTER_NONE, theta null and
// nang 1 (C = I).  Images are [pix][12] and per-angle images [a][pix][12] float32.
struct FoldJob {
    const float* raw;       // the primal paths' raw image
    const float* target;    // the L2 target
    const float* dimage;    // the image adjoint dg/dI
    float* image;           // the filtered images out
    float* dS;              // the adjoint input out
    const float* S_adj;     // the adjoint paths' raw image
    const float* theta;     // [nang] filter angles, or null
    float* dtheta;          // [nang] angle gradients, added into
    long long npix;
    int filter, nang;
};
constexpr int kMaxFoldJobs = 64;
int fold_launches(int njobs);
cudaError_t launch_apply_filter(const FoldJob* jobs, int njobs, cudaStream_t st);
cudaError_t launch_filter_adjoint_input(const FoldJob* jobs, int njobs, cudaStream_t st);
cudaError_t launch_theta_grad(const FoldJob* jobs, int njobs, cudaStream_t st);
cudaError_t launch_l2_loss(const FoldJob* jobs, int njobs, double scale, double* loss, cudaStream_t st);
cudaError_t launch_l2_adjoint_input(const FoldJob* jobs, int njobs, float scale2, cudaStream_t st);
cudaError_t launch_l2_theta_grad(const FoldJob* jobs, int njobs, float scale2, cudaStream_t st);
}  // namespace dppt
