// Wavefront schedule of the same path tracer: the megakernel's per-vertex work
// split into stage kernels over compacted lists of live paths,
//   extend  (closest hit)  ->  shade (surface data, light and BSDF samples)
//   -> shadow (any hit of the light samples) -> finish (per-vertex action,
//   next ray), the finish stage launched once per pass so that cache passes
//   and dual-number replays run in separate, coherent kernels.
// Path state, hits and the per-vertex cache of E_i / W_i live in the context
// workspace ([vertex][component][path] for the cache, so that a warp's loads
// are contiguous).  The replay re-traces the path with the same stage code
// and Philox counters as the cache pass.  Every stage reads its list length
// from device memory, so a wave is a fixed sequence of launches.
#include "trace.cuh"

namespace dppt {

struct __align__(16) WfPath {
    Walk w;
    unsigned long long pid;
    float a[3][4];
    float raw[12];
    int job, phase, n, i;
};
struct __align__(16) WfVertex {
    VCtx vc;
    NeePending ne;
    Shade sh;
    int hit, visible;
};

struct WfLists {
    int* l0;      // live paths in the cache pass
    int* l1;      // live paths in the replay pass
    int* next0;
    int* next1;
    int* shadow;
    int* count;   // [0] n0, [1] n1, [2] next0, [3] next1, [4] shadow
};

__device__ __forceinline__ int list_at(const WfLists& L, int idx) {
    int n0 = L.count[0];
    return idx < n0 ? L.l0[idx] : L.l1[idx - n0];
}

__global__ void k_wf_init(const DScene S, const __grid_constant__ JobTable T, int job, long long p0, int nq,
                          WfPath* paths, WfLists L) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const DJob& J = T.job[job];
    WfPath& st = paths[q];
    st.pid = (unsigned long long)(p0 + q);
    st.job = job;
    st.phase = 0;
    st.n = 0;
    st.i = 0;
    walk_begin(S, J, st.pid, (long long)(st.pid / J.spp), st.w);
    L.l0[q] = q;
    if (q == 0) { L.count[0] = nq; L.count[1] = 0; }
}

__global__ void k_wf_extend(const DScene S, WfPath* paths, WfVertex* vtx, HitRec* hits, WfLists L, unsigned* status) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.count[0] + L.count[1]) return;
    int q = list_at(L, idx);
    const Walk& w = paths[q].w;
    HitRec h;
    vtx[q].hit = trace_closest<false>(S, w.o, w.d, h, status, nullptr) ? 1 : 0;
    hits[q] = h;
}

__global__ void k_wf_shade(const DScene S, const DParams P, const __grid_constant__ JobTable T, WfPath* paths,
                           WfVertex* vtx, const HitRec* hits, WfLists L) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.count[0] + L.count[1]) return;
    int q = list_at(L, idx);
    WfVertex& V = vtx[q];
    if (!V.hit) return;
    const WfPath& st = paths[q];
    walk_shade(S, P, T.job[st.job], st.pid, st.w, hits[q], V.vc, V.ne, V.sh);
    V.visible = 0;
    if (V.ne.state == 1) L.shadow[atomicAdd(L.count + 4, 1)] = q;
}

__global__ void k_wf_shadow(const DScene S, WfVertex* vtx, WfLists L, unsigned* status) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.count[4]) return;
    int q = L.shadow[idx];
    const NeePending& ne = vtx[q].ne;
    vtx[q].visible = trace_any<false>(S, ne.o2, ne.dir, ne.tmax, status, nullptr) ? 0 : 1;
}

// Finish stage for the paths of one pass (phase 0: cache pass, phase 1: replay).
template <int MODE>
__global__ void k_wf_finish(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T,
                            WfPath* paths, WfVertex* vtx, float* cache, long long Q, int cap, WfLists L, int phase,
                            float* rawp, unsigned* sig) {
    extern __shared__ float sgrad[];
    const int nscal = (MODE == 1 && phase == 1) ? S.num_ior + S.num_sheets + 12 * S.num_lights : 0;
    for (int k = threadIdx.x; k < nscal; k += blockDim.x) sgrad[k] = 0.0f;
    if (nscal) __syncthreads();
    const int count = phase == 0 ? L.count[0] : L.count[1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < count) {
        const int q = phase == 0 ? L.l0[idx] : L.l1[idx];
        WfPath& st = paths[q];
        const DJob& J = T.job[st.job];
        PathVis<GlobalCache> vis;
        vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad;
        vis.C.base = cache; vis.C.Q = Q; vis.C.q = q; vis.C.cap = cap;
        vis.n = st.n; vis.i = st.i; vis.phase = st.phase;
        if (phase == 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < 4; ++k) vis.a[c][k] = st.a[c][k];
        }
        WfVertex& V = vtx[q];
        bool cont = false;
        if (V.hit) cont = walk_finish(S, P, st.w, V.vc, V.ne, V.visible != 0, V.sh, vis);
        bool done = false;
        if (cont) {
            if (phase == 0) L.next0[atomicAdd(L.count + 2, 1)] = q;
            else L.next1[atomicAdd(L.count + 3, 1)] = q;
        } else if (phase == 0) {
            float L0[12];
            vis.fold(L0);
            Rot<float> Rc = camera_rot(S.cams[J.cam], st.w.d1);
            const float inv = 1.0f / (float)J.spp;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
                rot_apply(Rc, v);
#pragma unroll
                for (int k = 0; k < 4; ++k) st.raw[4 * c + k] = v[k] * inv;
            }
            if (MODE == 1 && vis.n > 0) {
                const long long pix = (long long)(st.pid / J.spp);
                const float* ds = J.dS + pix * 12;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float av[4] = {__ldg(ds + 4 * c) * inv, __ldg(ds + 4 * c + 1) * inv,
                                   __ldg(ds + 4 * c + 2) * inv, __ldg(ds + 4 * c + 3) * inv};
                    rot_apply_row(Rc, av);
#pragma unroll
                    for (int k = 0; k < 4; ++k) vis.a[c][k] = av[k];
                }
                vis.phase = 1;
                vis.i = 0;
                walk_begin(S, J, st.pid, pix, st.w);
                L.next1[atomicAdd(L.count + 3, 1)] = q;
            } else {
                done = true;
            }
        } else {
            done = true;
        }
        st.n = vis.n; st.i = vis.i; st.phase = vis.phase;
        if (MODE == 1 && vis.phase == 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < 4; ++k) st.a[c][k] = vis.a[c][k];
        }
        if (done) {
            float4* o = reinterpret_cast<float4*>(rawp + (long long)q * 12);
            o[0] = make_float4(st.raw[0], st.raw[1], st.raw[2], st.raw[3]);
            o[1] = make_float4(st.raw[4], st.raw[5], st.raw[6], st.raw[7]);
            o[2] = make_float4(st.raw[8], st.raw[9], st.raw[10], st.raw[11]);
            if (sig) sig[q] = fnv(st.w.sig, (unsigned)st.w.nv);
        }
    }
    if (nscal) {
        __syncthreads();
        float* gdst[3] = {G.ior, G.sheet, G.le};
        const int nI = S.num_ior, nS = S.num_sheets;
        for (int k = threadIdx.x; k < nscal; k += blockDim.x) {
            float v = sgrad[k];
            if (v == 0.0f) continue;
            float* base;
            int off;
            if (k < nI) { base = gdst[0]; off = k; }
            else if (k < nI + nS) { base = gdst[1]; off = k - nI; }
            else { base = gdst[2]; off = k - nI - nS; }
            if (base) atomicAdd(base + off, v);
        }
    }
}

// next lists become the live lists; the paths' raw values of a finished wave are summed per pixel
__global__ void k_wf_swap(WfLists L) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        L.count[0] = L.count[2];
        L.count[1] = L.count[3];
        L.count[2] = 0;
        L.count[3] = 0;
        L.count[4] = 0;
    }
}

__global__ void k_wf_pixels(const float* rawp, int spp, long long npix, float* dst) {
    long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0f;
    for (int s = 0; s < spp; ++s) {
        const float4* r = reinterpret_cast<const float4*>(rawp + (pix * spp + s) * 12);
        for (int qd = 0; qd < 3; ++qd) {
            float4 t = r[qd];
            acc[4 * qd] += t.x; acc[4 * qd + 1] += t.y; acc[4 * qd + 2] += t.z; acc[4 * qd + 3] += t.w;
        }
    }
    float4* o = reinterpret_cast<float4*>(dst + pix * 12);
    o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    o[2] = make_float4(acc[8], acc[9], acc[10], acc[11]);
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

size_t wavefront_bytes(long long Q, int cap) {
    size_t b = 0;
    b += align_up(sizeof(WfPath) * Q);
    b += align_up(sizeof(WfVertex) * Q);
    b += align_up(sizeof(HitRec) * Q);
    b += align_up(sizeof(float) * 12 * Q);            // raw per path
    b += 5 * align_up(sizeof(int) * Q);               // lists
    b += align_up(sizeof(int) * 8);
    b += align_up(sizeof(float) * 31 * (size_t)cap * Q);
    return b;
}

// Renders (mode 0) or differentiates (mode 1) job `job` of the table in waves of
// at most Q paths (whole pixels), writing the per-pixel raw image to J.raw.
cudaError_t run_wavefront(int mode, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, int job,
                          void* ws, long long Q, int cap, int block, unsigned* status, cudaStream_t st,
                          StageLog* log) {
    const DJob& J = T.job[job];
    char* p = static_cast<char*>(ws);
    WfPath* paths = reinterpret_cast<WfPath*>(p); p += align_up(sizeof(WfPath) * Q);
    WfVertex* vtx = reinterpret_cast<WfVertex*>(p); p += align_up(sizeof(WfVertex) * Q);
    HitRec* hits = reinterpret_cast<HitRec*>(p); p += align_up(sizeof(HitRec) * Q);
    float* rawp = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 12 * Q);
    int* lists[5];
    for (int k = 0; k < 5; ++k) { lists[k] = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * Q); }
    int* count = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * 8);
    float* cache = reinterpret_cast<float*>(p);
    const long long npix = (long long)J.W * J.H;
    const long long pix_per_wave = std::max(1LL, Q / J.spp);
    const int passes = mode == 1 ? 2 : 1;
    const size_t smem = mode == 1 ? sizeof(float) * (size_t)(S.num_ior + S.num_sheets + 12 * S.num_lights) : 0;
    for (long long pix0 = 0; pix0 < npix; pix0 += pix_per_wave) {
        const long long wp = std::min(pix_per_wave, npix - pix0);
        const int nq = (int)(wp * J.spp);
        const int grid = (nq + block - 1) / block;
        WfLists A{lists[0], lists[1], lists[2], lists[3], lists[4], count};
        cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * 8, st);
        if (e != cudaSuccess) return e;
        int tok = log->begin(kStageWfInit, st);
        k_wf_init<<<grid, block, 0, st>>>(S, T, job, pix0 * J.spp, nq, paths, A);
        log->end(tok, st);
        for (int it = 0; it < passes * J.depth; ++it) {
            // lists alternate between two buffer pairs: the next lists of one iteration are the
            // live lists of the following one (k_wf_swap moves the counts)
            WfLists L = (it & 1) ? WfLists{lists[2], lists[3], lists[0], lists[1], lists[4], count} : A;
            unsigned* sg = J.sig ? J.sig + pix0 * J.spp : nullptr;
            tok = log->begin(kStageWfExtend, st);
            k_wf_extend<<<grid, block, 0, st>>>(S, paths, vtx, hits, L, status);
            log->end(tok, st);
            tok = log->begin(kStageWfShade, st);
            k_wf_shade<<<grid, block, 0, st>>>(S, P, T, paths, vtx, hits, L);
            log->end(tok, st);
            tok = log->begin(kStageWfShadow, st);
            k_wf_shadow<<<grid, block, 0, st>>>(S, vtx, L, status);
            log->end(tok, st);
            tok = log->begin(kStageWfCache, st);
            if (mode == 0) k_wf_finish<0><<<grid, block, 0, st>>>(S, P, G, T, paths, vtx, cache, Q, cap, L, 0, rawp, sg);
            else k_wf_finish<1><<<grid, block, 0, st>>>(S, P, G, T, paths, vtx, cache, Q, cap, L, 0, rawp, sg);
            log->end(tok, st);
            if (mode == 1) {
                tok = log->begin(kStageWfReplay, st);
                k_wf_finish<1><<<grid, block, smem, st>>>(S, P, G, T, paths, vtx, cache, Q, cap, L, 1, rawp, sg);
                log->end(tok, st);
            }
            tok = log->begin(kStageWfSwap, st);
            k_wf_swap<<<1, 32, 0, st>>>(L);
            log->end(tok, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (J.raw) {
            tok = log->begin(kStageWfPixels, st);
            k_wf_pixels<<<(int)((wp + 127) / 128), 128, 0, st>>>(rawp, J.spp, wp, J.raw + pix0 * 12);
            log->end(tok, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace dppt
