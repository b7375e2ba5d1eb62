// Wavefront schedule of the same path tracer: the megakernel's per-vertex work split into
// stage kernels over compacted lists of live paths.  A cache-pass iteration runs
//   extend + shade (closest hit, then surface data, light and BSDF samples; one kernel,
//   or two with DPPT_WF_FUSE_SHADE=0) -> shadow (any hit of the light samples)
//   -> cache (per-vertex action, next ray);
// the replay runs in the same iterations as one kernel per material type, over the paths
// binned by the type of their next vertex: it shades that vertex itself from the hit and
// light-sample visibility the cache pass stored (no traversal, no vertex record) and
// evaluates it with dual numbers, with the same code and Philox counters as the cache
// pass.  Path state lives in the context workspace as per-path records that one thread
// moves with float4 loads and stores, each aligned so that it fills whole 64-byte blocks:
// the lists' order scatters a warp's paths over the wave, so a thread's record, not a
// warp's, is the unit of memory traffic.  The path's state (walk 64 B, adjoint row 48 B,
// bookkeeping 16 B) is one 128-byte record, the vertex handed from shade to cache another;
// the per-vertex cache holds one 144-byte record per (vertex, path), whole whatever
// fraction of the wave's paths is still live.  Every stage reads its list length from
// device memory and loops over it with a grid stride, so a wave is a fixed sequence of
// launches.
#include <algorithm>
#include <vector>

#include "wavefront.cuh"

// resident threads per SM the traversal kernels' register allocation must allow (as blocks
// of the largest wavefront block size, 512)
#ifndef DPPT_WF_TRAVERSE_MIN_BLOCKS
#define DPPT_WF_TRAVERSE_MIN_BLOCKS 2
#endif
// resident 128-thread blocks per SM the finish kernels' register allocation must allow
// (4 -> at most 128 registers per thread, 3 -> at most 168); chosen by measured sweeps
#ifndef DPPT_WF_CACHE_MIN_BLOCKS
#define DPPT_WF_CACHE_MIN_BLOCKS 4
#endif
#ifndef DPPT_WF_REPLAY_MIN_BLOCKS
#define DPPT_WF_REPLAY_MIN_BLOCKS 4
#endif
// the same for the replay kernel of diffuse vertices, the simplest material (5 -> at most
// 102 registers)
#ifndef DPPT_WF_REPLAY_DIFFUSE_MIN_BLOCKS
#define DPPT_WF_REPLAY_DIFFUSE_MIN_BLOCKS 4
#endif
// resident 512-thread blocks per SM the fused extend + shade kernel's registers must allow
#ifndef DPPT_WF_EXTEND_SHADE_MIN_BLOCKS
#define DPPT_WF_EXTEND_SHADE_MIN_BLOCKS 2
#endif
// extend and shade fused in one kernel (1) or as two launches (0)
#ifndef DPPT_WF_FUSE_SHADE
#define DPPT_WF_FUSE_SHADE 1
#endif
// resident 512-thread blocks per SM the shade kernel's register allocation must allow
// (2 -> at most 64 registers per thread)
#ifndef DPPT_WF_SHADE_MIN_BLOCKS
#define DPPT_WF_SHADE_MIN_BLOCKS 2
#endif

namespace dppt {
__global__ void k_wf_init(const DScene S, const __grid_constant__ JobTable T, const __grid_constant__ WaveTable wt,
                          WfState W, WfLists L) {
    const int stride = gridDim.x * blockDim.x;
    const int nq = (int)wt.nq;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
        Walk w;
        wave_start_path(S, T, wt, q, W, w);
        L.l0[q] = q;
        if (q == 0) L.cur[0] = nq;
    }
}

// The traversal stack of the wavefront's traversal kernels: its top in shared memory (the
// launch passes trav_stack_smem(block) bytes of dynamic shared memory), unless
// DPPT_TRAV_SHARED_STACK is 0.
using WfStack = std::conditional<(DPPT_TRAV_SHARED_STACK > 0), SharedStack, LocalStack>::type;
__device__ __forceinline__ void stack_init(LocalStack&) {}
__device__ __forceinline__ void stack_init(SharedStack& st) {
    extern __shared__ int trav_sh[];
    st.sh = trav_sh + threadIdx.x;
}

// Closest hits of the live paths, one ray per thread in a grid-stride loop.  The list
// keeps the samples of a pixel together, so a warp's rays share their origin.  Only the
// cache pass traces: the replay reads its hits from the cache (kWfHitComp).
__global__ void __launch_bounds__(512, DPPT_WF_TRAVERSE_MIN_BLOCKS)
k_wf_extend(const DScene S, WfState W, WfLists L, unsigned* status) {
    const int n = L.cur[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        L.nxt[0] = 0; L.cur[4] = 0;
        for (int b = 8; b < 16; ++b) L.nxt[b] = 0;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const int q = L.l0[idx];
        const float4 a = W.path[q].a, b = W.path[q].b;
        HitRec h;
        WfStack stk;
        stack_init(stk);
        const bool hit = trace_closest_with<false>(S, f3{a.x, a.y, a.z}, f3{b.x, b.y, b.z}, h, status, nullptr, stk);
        W.hit[q] = hit ? make_float4(h.t, h.b1, h.b2, __int_as_float(code_of(S, true, h)))
                       : make_float4(0.f, 0.f, 0.f, __int_as_float(code_of(S, false, h)));
    }
}


// Surface data, light sample and BSDF sample of each cache-pass path's new vertex; in the
// adjoint (store_hits) the hit is also stored in the cache at the vertex's slot for the
// replay.
template <bool NM>
__global__ void __launch_bounds__(512, DPPT_WF_SHADE_MIN_BLOCKS)
k_wf_shade(const DScene S, const DParams P, const __grid_constant__ JobTable T, WfState W, WfLists L,
           int store_hits) {
    const int n = L.cur[0];
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const int q = L.l0[idx];
        const float4 hv = W.hit[q];
        const bool miss = __float_as_int(hv.w) == kMissCode;
        if (store_hits) {
            const int v = __float_as_int(W.path[q].c.w) & 0xff;     // the vertex's slot (see put_walk)
            float* rec = W.hit_rec(v - 1, q);
            *reinterpret_cast<float4*>(rec + W.hit_comp) = hv;
            if (miss && W.vis_comp >= 0) rec[W.vis_comp] = __int_as_float(kBinMiss << 1);
        }
        if (miss) {
            W.vtx[q].ids = make_int4(0, 0, 0, 0);
            continue;
        }
        HitRec h;
        decode_hit(S, hv, h);
        Walk w;
        get_walk(W.path + q, w);
        const WfMeta m = W.path[q].meta;
        const unsigned long long pid = (unsigned long long)m.lo | ((unsigned long long)m.hi << 32);
        VCtx vc;
        NeePending ne;
        Shade sh;
        walk_shade<NM>(S, P, T.job[m.job], pid, w, h, vc, ne, sh);
        put_vertex(W.vtx + q, vc, ne, sh);
        if (ne.state == 1) {
            W.ray[q] = WfRay{make_float4(ne.o2.x, ne.o2.y, ne.o2.z, ne.tmax), make_float4(ne.dir.x, ne.dir.y, ne.dir.z, 0.f)};
            L.shadow[atomicAdd(L.cur + 4, 1)] = q;
        }
        W.visible[q] = 0;
    }
}

// Extend and shade in one kernel: the closest hit of each cache-pass path and, from it in
// registers, the vertex's surface data and samples.  The launch's block 0 zeroes the
// counts the iteration appends to after this kernel and the next iteration's shadow
// count (this kernel appends to this iteration's, zeroed one iteration earlier).  The
// first iteration of a wave (FIRST) starts the wave's paths itself (camera rays, path
// records and the identity cache-pass list), from the wave's pieces of jobs.
template <bool NM, bool FIRST>
__global__ void __launch_bounds__(512, DPPT_WF_EXTEND_SHADE_MIN_BLOCKS)
k_wf_extend_shade(const DScene S, const DParams P, const __grid_constant__ JobTable T, WfState W, WfLists L,
                  int store_hits, unsigned* status, const __grid_constant__ WaveTable wt) {
    const int nq = (int)wt.nq;
    const int n = FIRST ? nq : L.cur[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        L.nxt[0] = 0; L.nxt[4] = 0;
        for (int b = 8; b < 16; ++b) L.nxt[b] = 0;
        if (FIRST) L.cur[0] = nq;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const int q = FIRST ? idx : L.l0[idx];
        HitRec h;
        bool hit;
        Walk w;
        WfStack stk;
        stack_init(stk);
        if (FIRST) {
            wave_start_path(S, T, wt, q, W, w);
            L.l0[q] = q;
            hit = trace_closest_with<false>(S, w.o, w.d, h, status, nullptr, stk);
        } else {
            {
                const float4 a = W.path[q].a, b = W.path[q].b;
                hit = trace_closest_with<false>(S, f3{a.x, a.y, a.z}, f3{b.x, b.y, b.z}, h, status, nullptr, stk);
            }
            get_walk(W.path + q, w);
        }
        if (store_hits) {
            float* rec = W.hit_rec(w.v - 1, q);
            const int code = code_of(S, hit, h);
            *reinterpret_cast<float4*>(rec + W.hit_comp) =
                hit ? make_float4(h.t, h.b1, h.b2, __int_as_float(code)) : make_float4(0.f, 0.f, 0.f, __int_as_float(code));
            if (!hit && W.vis_comp >= 0) rec[W.vis_comp] = __int_as_float(kBinMiss << 1);
        }
        if (!hit) {
            W.vtx[q].ids = make_int4(0, 0, 0, 0);
            continue;
        }
        if (h.prim >= S.num_tris) h.slot = -1;
        const WfMeta m = W.path[q].meta;
        const unsigned long long pid = (unsigned long long)m.lo | ((unsigned long long)m.hi << 32);
        VCtx vc;
        NeePending ne;
        Shade sh;
        walk_shade<NM>(S, P, T.job[m.job], pid, w, h, vc, ne, sh);
        put_vertex(W.vtx + q, vc, ne, sh);
        if (ne.state == 1) {
            W.ray[q] = WfRay{make_float4(ne.o2.x, ne.o2.y, ne.o2.z, ne.tmax), make_float4(ne.dir.x, ne.dir.y, ne.dir.z, 0.f)};
            L.shadow[atomicAdd(L.cur + 4, 1)] = q;
        }
        W.visible[q] = 0;
    }
}

__global__ void __launch_bounds__(512, DPPT_WF_TRAVERSE_MIN_BLOCKS)
k_wf_shadow(const DScene S, WfState W, WfLists L, unsigned* status) {
    const int n = L.cur[4];
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const int q = L.shadow[idx];
        const WfRay r = W.ray[q];
        WfStack stk;
        stack_init(stk);
        W.visible[q] = trace_any_with<false>(S, f3{r.o_tmax.x, r.o_tmax.y, r.o_tmax.z}, f3{r.dir.x, r.dir.y, r.dir.z},
                                             r.o_tmax.w, status, nullptr, stk) ? 0 : 1;
    }
}

// Per-vertex action of one pass.  PHASE 0 (cache pass): cache E_i / W_i; at the end of
// the walk fold the cache, store the path's raw Stokes value and, for the adjoint (MODE
// 1), start the replay.  PHASE 1: the replay of replay bin BIN (MODE 1 only), compiled for
// material type MT (-1: any).  It shades its vertex itself from the cached hit and light-
// sample visibility (no vertex record, no traversal) and appends each continuing path to
// the bin of its next vertex.
template <int MODE, int PHASE, bool NM, int MT = -1, int BIN = -1>
__global__ void __launch_bounds__(128, PHASE == 0 ? DPPT_WF_CACHE_MIN_BLOCKS
                                                  : MT == DPPT_MAT_DIFFUSE ? DPPT_WF_REPLAY_DIFFUSE_MIN_BLOCKS
                                                                           : DPPT_WF_REPLAY_MIN_BLOCKS)
k_wf_finish(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T, WfState W, WfLists L) {
    extern __shared__ float sgrad[];
    if (PHASE == 1) sgrad_zero(S, sgrad);
    static_assert(PHASE == 0 || BIN >= 0, "the replay runs over one bin");
    // the pass's list: the cache list or one replay bin
    const int* list = PHASE == 0 ? L.l0 : L.bins + (long long)(BIN < 0 ? 0 : BIN) * L.binQ;
    const int count = PHASE == 0 ? L.cur[0] : L.cur[8 + (BIN < 0 ? 0 : BIN)];
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += stride) {
        const int q = list[idx];
        const WfMeta m = W.path[q].meta;
        const DJob& J = T.job[m.job];
        Walk w;
        get_walk(W.path + q, w);
        PathVis<GlobalCache, MT, NM> vis;
        vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad;
        vis.C.base = W.cache; vis.C.Q = W.Q; vis.C.q = q; vis.C.cap = W.cap; vis.C.stride = W.rec_floats;
        vis.n = (m.pni >> 8) & 0xff; vis.i = (m.pni >> 16) & 0xff; vis.phase = PHASE;
        vis.has_last = false;          // set, and consumed by the fold, within this launch
        vis.adjoint = MODE == 1;
        VCtx vc;
        NeePending ne;
        Shade sh;
        bool cont = false;
        if (PHASE == 0) {
            if (get_vertex(W.vtx + q, w, vc, ne, sh)) {
                if (NM) apply_normal_map(S, P, vc);
                const int visible = W.visible[q];
                const int slot = w.v - 1;
                cont = walk_finish(S, P, w, vc, ne, visible != 0, sh, vis);
                // the replay reads it back; stored after walk_finish, whose cache write zeroes it
                if (MODE == 1)
                    W.rec(slot, q)[kWfVisComp] = __int_as_float(replay_bin(S, vc.mat) << 1 | (visible != 0 ? 1 : 0));
            }
        } else {
            const float4 hv = *reinterpret_cast<const float4*>(W.rec(w.v - 1, q) + W.hit_comp);
            if (__float_as_int(hv.w) != kMissCode) {
                HitRec h;
                decode_hit(S, hv, h);
                const unsigned long long pid = (unsigned long long)m.lo | ((unsigned long long)m.hi << 32);
                walk_shade<NM, MT>(S, P, J, pid, w, h, vc, ne, sh);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float4 r = W.path[q].arow[c];
                    vis.a[c][0] = r.x; vis.a[c][1] = r.y; vis.a[c][2] = r.z; vis.a[c][3] = r.w;
                }
                cont = walk_finish(S, P, w, vc, ne, (W.vis_word(w.v - 1, q) & 1) != 0, sh, vis);
            }
        }
        bool done = false;
        int phase = PHASE;
        if (cont && PHASE == 1) {
            const int b = replay_bin_of(W, q, w.v - 1);
            if (b == kBinMiss) done = true;     // the next ray left the scene: nothing to replay
            else bin_append(L, b, q);
        } else if (cont) {
            L.next0[atomicAdd(L.nxt + 0, 1)] = q;
        } else if (PHASE == 0) {
            float L0[12];
            vis.fold(L0);
            Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
            const float inv = 1.0f / (float)J.spp;
            float rv[12];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
                rot_apply(Rc, v);
#pragma unroll
                for (int k = 0; k < 4; ++k) rv[4 * c + k] = v[k] * inv;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
                W.raw[3 * (long long)q + c] = make_float4(rv[4 * c], rv[4 * c + 1], rv[4 * c + 2], rv[4 * c + 3]);
            if (MODE == 1 && vis.n > 0) {
                const unsigned long long pid = (unsigned long long)m.lo | ((unsigned long long)m.hi << 32);
                const long long pix = (long long)(pid / J.spp);
                const float* ds = J.dS + pix * 12;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float av[4] = {__ldg(ds + 4 * c) * inv, __ldg(ds + 4 * c + 1) * inv,
                                   __ldg(ds + 4 * c + 2) * inv, __ldg(ds + 4 * c + 3) * inv};
                    rot_apply_row(Rc, av);
                    W.path[q].arow[c] = make_float4(av[0], av[1], av[2], av[3]);
                }
                phase = 1;
                vis.i = 0;
                walk_begin(S, J, pid, pix, w);
                bin_append(L, replay_bin_of(W, q, 0), q);
            } else {
                done = true;
            }
        } else {
            done = true;
        }
        if (PHASE == 1 && !done) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                W.path[q].arow[c] = make_float4(vis.a[c][0], vis.a[c][1], vis.a[c][2], vis.a[c][3]);
        }
        if (done) {
            if (J.sig) J.sig[(unsigned long long)m.lo | ((unsigned long long)m.hi << 32)] = fnv(w.sig, (unsigned)w.nv);
        } else {
            W.path[q].meta.pni = phase | (vis.n << 8) | (vis.i << 16);
            put_walk(W.path + q, w);
        }
    }
    if (PHASE == 1) sgrad_flush(S, G, sgrad);
}

// sums the spp paths of each pixel of a finished wave (deterministic order) into the raw
// image of the pixel's job, when it has one
__global__ void k_wf_pixels(const float4* raw, const __grid_constant__ JobTable T, const __grid_constant__ WaveTable wt) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= wt.npix) return;
    const WaveSeg& sg = wt.seg[wave_piece_of_pixel(wt, i)];
    const DJob& J = T.job[sg.job];
    if (!J.raw) return;
    const long long local = i - sg.qpix0;
    const float4* r = raw + 3 * (sg.q0 + local * J.spp);
    float4 acc[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    for (int s = 0; s < J.spp; ++s)
        for (int c = 0; c < 3; ++c) {
            const float4 t = r[3 * s + c];
            acc[c].x += t.x; acc[c].y += t.y; acc[c].z += t.z; acc[c].w += t.w;
        }
    float4* o = reinterpret_cast<float4*>(J.raw + (sg.pix0 + local) * 12);
    o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// the hybrid replay's per-path arrays (HybWs): block data, route bytes, flag words
static int hyb_blocks(int cap, int k) { return cap / k + 2; }
static int hyb_route_stride(int cap) { return (cap + 15) & ~15; }

size_t wavefront_bytes(long long Q, int cap, int k) {
    size_t b = 0;
    b += align_up(sizeof(WfPath) * Q);
    b += align_up(sizeof(WfVtx) * Q);
    b += align_up(sizeof(float4) * Q);          // hits
    b += align_up(sizeof(WfRay) * Q);
    b += align_up(sizeof(int) * Q);             // visible
    b += align_up(sizeof(float4) * 3 * Q);      // raw per path
    b += 3 * align_up(sizeof(int) * Q);         // lists
    b += align_up(sizeof(int) * 32);
    b += 2 * align_up(sizeof(int) * 8 * Q);     // replay bins of this and the next iteration
    if (k <= 1) {
        b += align_up(sizeof(float) * kWfCacheComps * (size_t)cap * Q);
    } else {
        const int nb = hyb_blocks(cap, k), fw = (nb + 31) / 32;
        b += align_up(sizeof(float4) * (size_t)cap * Q);            // hits
        b += align_up((size_t)cap * Q);                              // light-sample visibility
        b += align_up(sizeof(float) * 60 * (size_t)nb * Q);          // block data
        b += align_up((size_t)hyb_route_stride(cap) * Q);            // routes
        b += align_up(sizeof(float) * 31 * (size_t)k * Q);           // look-ahead
        b += align_up(sizeof(float) * 60 * Q);                       // replay's block throughput + emission
        b += align_up(sizeof(unsigned) * (size_t)fw * Q);            // recomputed-block flags
    }
    return b;
}

// The replay of bin MT with the kernel compiled for that material type.
struct ReplayArgs {
    const DScene& S;
    const DParams& P;
    const DGrads& G;
    const JobTable& T;
    const WfState& W;
    const WfLists& L;
    int grid;
    size_t smem;
    cudaStream_t st;
    bool nmaps;
};
template <int MT>
static void launch_replay_bin(const ReplayArgs& a) {
    if (a.nmaps) k_wf_finish<1, 1, true, MT, MT><<<a.grid, 128, a.smem, a.st>>>(a.S, a.P, a.G, a.T, a.W, a.L);
    else k_wf_finish<1, 1, false, MT, MT><<<a.grid, 128, a.smem, a.st>>>(a.S, a.P, a.G, a.T, a.W, a.L);
}
// One replay iteration: a kernel per binned material type present, then the other bin when
// the scene has a type without a kernel of its own.  The bins hold disjoint paths, so with a
// side stream the first bin runs on the launching stream and every other bin on the side
// stream beside it: the small bins are latency-bound on few paths and would otherwise run
// one after another.
static void replay_iteration(const ReplayArgs& ra, unsigned types, const SideStream* side, StageLog* log) {
    const bool other = (types & ~kBinnedTypes) != 0;
    const int nbins = (other ? 1 : 0) + __builtin_popcount(types & kBinnedTypes);
    const int tok = log->begin(kStageWfReplay, ra.st, nbins);
    const bool fork = side && nbins > 1;
    ReplayArgs rs = ra;
    if (fork) {
        cudaEventRecord(side->fork, ra.st);
        cudaStreamWaitEvent(side->st, side->fork, 0);
        rs.st = side->st;
    }
    int k = 0;   // bins launched so far: the first on the launching stream
    auto bin = [&](int t, void (*launch)(const ReplayArgs&)) {
        if (types & (1u << t)) launch(k++ == 0 ? ra : rs);
    };
    bin(DPPT_MAT_DIFFUSE, launch_replay_bin<DPPT_MAT_DIFFUSE>);
    bin(DPPT_MAT_CONDUCTOR_GGX, launch_replay_bin<DPPT_MAT_CONDUCTOR_GGX>);
    bin(DPPT_MAT_PLASTIC_GGX, launch_replay_bin<DPPT_MAT_PLASTIC_GGX>);
    bin(DPPT_MAT_SMOOTH_DIELECTRIC, launch_replay_bin<DPPT_MAT_SMOOTH_DIELECTRIC>);
    bin(DPPT_MAT_POLARIZER_SHEET, launch_replay_bin<DPPT_MAT_POLARIZER_SHEET>);
    bin(DPPT_MAT_RETARDER_SHEET, launch_replay_bin<DPPT_MAT_RETARDER_SHEET>);
    bin(DPPT_MAT_EMITTER, launch_replay_bin<DPPT_MAT_EMITTER>);
    if (other) {
        const ReplayArgs& ro = k++ == 0 ? ra : rs;
        if (ro.nmaps) k_wf_finish<1, 1, true, -1, kBinOther><<<ro.grid, 128, ro.smem, ro.st>>>(ro.S, ro.P, ro.G, ro.T, ro.W, ro.L);
        else k_wf_finish<1, 1, false, -1, kBinOther><<<ro.grid, 128, ro.smem, ro.st>>>(ro.S, ro.P, ro.G, ro.T, ro.W, ro.L);
    }
    if (fork) {
        cudaEventRecord(side->join, side->st);
        cudaStreamWaitEvent(ra.st, side->join, 0);
    }
    log->end(tok, ra.st);
}

// the forward-sweep megakernel of a cache-depth bucket
static cudaError_t launch_wf_sweep(int bucket, bool nmaps, const DScene& S, const DParams& P, const JobTable& T,
                                   const WaveTable& wt, const WfState& W, const WfLists& L, int block, unsigned* status,
                                   cudaStream_t st) {
    switch (bucket) {
        case 4: return launch_wf_sweep_4(nmaps, S, P, T, wt, W, L, block, status, st);
        case 8: return launch_wf_sweep_8(nmaps, S, P, T, wt, W, L, block, status, st);
        case 16: return launch_wf_sweep_16(nmaps, S, P, T, wt, W, L, block, status, st);
        case 32: return launch_wf_sweep_32(nmaps, S, P, T, wt, W, L, block, status, st);
        case 64: return launch_wf_sweep_64(nmaps, S, P, T, wt, W, L, block, status, st);
        case 128: return launch_wf_sweep_128(nmaps, S, P, T, wt, W, L, block, status, st);
        default: return cudaErrorInvalidValue;
    }
}

// The waves of a table's jobs: the jobs in order, each cut at pixel boundaries into pieces
// that fill waves of at most Q paths (a wave closes when the next pixel does not fit or it
// holds kMaxJobsPerLaunch pieces).  Q must hold one pixel of every job.
static std::vector<WaveTable> plan_waves(const JobTable& T, long long Q) {
    std::vector<WaveTable> waves;
    WaveTable cur{};
    for (int k = 0; k < T.njobs; ++k) {
        const DJob& J = T.job[k];
        const long long npix = (long long)J.W * J.H;
        long long pix = 0;
        while (pix < npix) {
            long long room = (Q - cur.nq) / J.spp;
            if (room == 0 || cur.nseg == kMaxJobsPerLaunch) {
                waves.push_back(cur);
                cur = WaveTable{};
                room = Q / J.spp;
            }
            const long long take = std::min(room, npix - pix);
            cur.seg[cur.nseg++] = WaveSeg{k, 0, pix, take, cur.nq, cur.npix};
            cur.nq += take * J.spp;
            cur.npix += take;
            cur.depth = std::max(cur.depth, J.depth);
            pix += take;
        }
    }
    if (cur.nseg > 0) waves.push_back(cur);
    return waves;
}

// Renders (mode 0) or differentiates (mode 1) every job of the table in waves of at most Q
// paths, several jobs sharing a wave, and writes each job's per-pixel raw image to J.raw.
cudaError_t run_wavefront(int mode, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,
                          void* ws, long long Q, int cap, int block, const WfHybrid& hy, int sweep, unsigned* status,
                          cudaStream_t st, const SideStream* side, StageLog* log) {
    char* p = static_cast<char*>(ws);
    WfState W;
    W.path = reinterpret_cast<WfPath*>(p); p += align_up(sizeof(WfPath) * Q);
    W.vtx = reinterpret_cast<WfVtx*>(p); p += align_up(sizeof(WfVtx) * Q);
    W.hit = reinterpret_cast<float4*>(p); p += align_up(sizeof(float4) * Q);
    W.ray = reinterpret_cast<WfRay*>(p); p += align_up(sizeof(WfRay) * Q);
    W.visible = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * Q);
    W.raw = reinterpret_cast<float4*>(p); p += align_up(sizeof(float4) * 3 * Q);
    int* lists[3];
    for (int k = 0; k < 3; ++k) { lists[k] = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * Q); }
    int* count = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * 32);
    int* bins[2];
    for (int k = 0; k < 2; ++k) { bins[k] = reinterpret_cast<int*>(p); p += align_up(sizeof(int) * 8 * Q); }
    W.cache = reinterpret_cast<float*>(p);
    W.Q = Q;
    W.cap = cap;
    W.rec_floats = kWfCacheComps; W.hit_comp = kWfHitComp; W.vis_comp = kWfVisComp; W.vis_plane = nullptr;
    const bool hyb = hy.k > 1;
    HybWs H{};
    if (hyb) {
        // hits instead of the per-vertex cache, then the hybrid visitor's per-path arrays
        W.rec_floats = 4; W.hit_comp = 0; W.vis_comp = -1;
        p += align_up(sizeof(float4) * (size_t)cap * Q);
        H.vis = reinterpret_cast<unsigned char*>(p); p += align_up((size_t)cap * Q);
        H.nb = hyb_blocks(cap, hy.k);
        H.fw = (H.nb + 31) / 32;
        H.rstride = hyb_route_stride(cap);
        H.ck = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 60 * (size_t)H.nb * Q);
        H.route = reinterpret_cast<unsigned char*>(p); p += align_up((size_t)H.rstride * Q);
        H.blk = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 31 * (size_t)hy.k * Q);
        H.btr = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * 60 * Q);
        H.flags = reinterpret_cast<unsigned*>(p);
        H.gamma = hy.gamma;
        H.eps = hy.eps;
    }
    const bool swp = mode == 1 && !hyb && sweep > 0;
    if (swp) {
        // the sweep's 64-byte records, then its plane of visibility words, in the cache's space
        W.rec_floats = kSweepRecFloats; W.hit_comp = kSweepHitComp; W.vis_comp = -1;
        W.vis_plane = reinterpret_cast<int*>(W.cache + (size_t)kSweepRecFloats * cap * Q);
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool nmaps = S.tri_tan != nullptr;   // the scene has normal maps: kernels with that path
    const unsigned types = (unsigned)S.mat_types;
    const int passes = mode == 1 ? 2 : 1;
    const size_t smem = mode == 1 ? sgrad_bytes(S) : 0;
    const size_t tsm = trav_stack_smem(block);   // the traversal kernels' shared stack tops
    for (const WaveTable& wt : plan_waves(T, Q)) {
        const int nq = (int)wt.nq;
        // stage kernels stride over their lists: a few resident waves of blocks at most
        const int grid = (int)std::min<long long>((nq + block - 1) / block, (long long)sms * (2048 / block));
        const int fgrid = (int)std::min<long long>((nq + 127) / 128, (long long)sms * DPPT_WF_CACHE_MIN_BLOCKS * 2);
        const WfLists A{lists[0], lists[1], lists[2], count, count + 16, bins[0], bins[1], (int)Q};
        const WfLists B{lists[1], lists[0], lists[2], count + 16, count, bins[1], bins[0], (int)Q};
        cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * 32, st);
        if (e != cudaSuccess) return e;
        int tok = 0;
        if (swp) {
            // the forward sweep in one megakernel; every path then starts its replay at the first
            // replay iteration, so depth iterations finish the wave
            tok = log->begin(kStageWfSweep, st);
            e = launch_wf_sweep(sweep, nmaps, S, P, T, wt, W, A, std::min(block, 256), status, st);
            log->end(tok, st);
            if (e != cudaSuccess) return e;
            for (int it = 1; it <= wt.depth; ++it) {
                const WfLists& L = (it & 1) ? B : A;
                if ((e = cudaMemsetAsync(L.nxt, 0, sizeof(int) * 16, st)) != cudaSuccess) return e;
                replay_iteration(ReplayArgs{S, P, G, T, W, L, fgrid, smem, st, nmaps}, types, side, log);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            tok = log->begin(kStageWfPixels, st);
            k_wf_pixels<<<(int)((wt.npix + 127) / 128), 128, 0, st>>>(W.raw, T, wt);
            log->end(tok, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            continue;
        }
#if !DPPT_WF_FUSE_SHADE
        tok = log->begin(kStageWfInit, st);
        k_wf_init<<<grid, block, 0, st>>>(S, T, wt, W, A);
        log->end(tok, st);
#endif
        for (int it = 0; it < passes * wt.depth; ++it) {
            // lists, counts and bins alternate between two buffers: the next ones of an
            // iteration are the live ones of the following iteration
            const WfLists& L = (it & 1) ? B : A;
            // While paths still run their cache pass, an iteration's replay (the paths that
            // finished theirs) runs on the side stream beside its shadow rays and cache pass:
            // the two touch disjoint paths and both append to the next iteration's bins with
            // atomics.  It starts after the iteration's extend launch, which zeroes the counts it
            // appends to, and joins before the next extend, which zeroes the counts it reads.
            const bool overlap = side && mode == 1 && !hyb && it > 0 && it < wt.depth;
            // a path's cache pass ends by iteration depth - 1 (one vertex per iteration), and no
            // path replays before iteration 1: the launches with nothing to do are skipped
            if (it >= wt.depth) {
                // what the extend launch would have zeroed: the counts appended to next
                if ((e = cudaMemsetAsync(L.nxt, 0, sizeof(int) * 16, st)) != cudaSuccess) return e;
            } else {
#if DPPT_WF_FUSE_SHADE
                tok = log->begin(kStageWfExtend, st);
                // the first iteration also starts the wave's paths
                if (it == 0) {
                    if (nmaps) k_wf_extend_shade<true, true><<<grid, block, tsm, st>>>(S, P, T, W, L, mode == 1, status, wt);
                    else k_wf_extend_shade<false, true><<<grid, block, tsm, st>>>(S, P, T, W, L, mode == 1, status, wt);
                } else {
                    if (nmaps) k_wf_extend_shade<true, false><<<grid, block, tsm, st>>>(S, P, T, W, L, mode == 1, status, wt);
                    else k_wf_extend_shade<false, false><<<grid, block, tsm, st>>>(S, P, T, W, L, mode == 1, status, wt);
                }
                log->end(tok, st);
#else
                tok = log->begin(kStageWfExtend, st);
                k_wf_extend<<<grid, block, tsm, st>>>(S, W, L, status);
                log->end(tok, st);
                tok = log->begin(kStageWfShade, st);
                if (nmaps) k_wf_shade<true><<<grid, block, 0, st>>>(S, P, T, W, L, mode == 1);
                else k_wf_shade<false><<<grid, block, 0, st>>>(S, P, T, W, L, mode == 1);
                log->end(tok, st);
#endif
                if (overlap) {
                    cudaEventRecord(side->fork, st);
                    cudaStreamWaitEvent(side->st, side->fork, 0);
                    replay_iteration(ReplayArgs{S, P, G, T, W, L, fgrid, smem, side->st, nmaps}, types, nullptr, log);
                }
                tok = log->begin(kStageWfShadow, st);
                k_wf_shadow<<<grid, block, tsm, st>>>(S, W, L, status);
                log->end(tok, st);
                tok = log->begin(kStageWfCache, st);
                if (hyb) {
                    if ((e = launch_wf_hybrid(0, hy.k, S, P, G, T, W, L, H, fgrid, 0, st)) != cudaSuccess) return e;
                } else if (mode == 0) {
                    if (nmaps) k_wf_finish<0, 0, true><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                    else k_wf_finish<0, 0, false><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                } else {
                    if (nmaps) k_wf_finish<1, 0, true><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                    else k_wf_finish<1, 0, false><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                }
                log->end(tok, st);
                if (overlap) {
                    cudaEventRecord(side->join, side->st);
                    cudaStreamWaitEvent(st, side->join, 0);
                }
            }
            if (mode == 1 && it > 0 && hyb) {
                tok = log->begin(kStageWfReplay, st);
                if ((e = launch_wf_hybrid(1, hy.k, S, P, G, T, W, L, H, fgrid, smem, st)) != cudaSuccess) return e;
                log->end(tok, st);
            } else if (mode == 1 && it > 0 && !overlap) {
                replay_iteration(ReplayArgs{S, P, G, T, W, L, fgrid, smem, st, nmaps}, types, side, log);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        tok = log->begin(kStageWfPixels, st);
        k_wf_pixels<<<(int)((wt.npix + 127) / 128), 128, 0, st>>>(W.raw, T, wt);
        log->end(tok, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dppt
