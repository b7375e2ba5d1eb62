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

#include "trace.cuh"

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
// resident 512-thread blocks per SM the shade kernel's register allocation must allow
// (2 -> at most 64 registers per thread)
// resident 512-thread blocks per SM the fused extend + shade kernel's registers must allow
#ifndef DPPT_WF_EXTEND_SHADE_MIN_BLOCKS
#define DPPT_WF_EXTEND_SHADE_MIN_BLOCKS 2
#endif
// extend and shade fused in one kernel (1) or as two launches (0)
#ifndef DPPT_WF_FUSE_SHADE
#define DPPT_WF_FUSE_SHADE 1
#endif
#ifndef DPPT_WF_SHADE_MIN_BLOCKS
#define DPPT_WF_SHADE_MIN_BLOCKS 2
#endif

namespace dppt {

struct __align__(16) WfMeta { unsigned lo, hi; int job, pni; };  // pid, job, phase | n << 8 | i << 16
// a path's state: walk (o, prev_pdf) (d, sig) (xprev, v | nv | delta) (d1, -), adjoint row
// (3 channels), bookkeeping
struct __align__(128) WfPath { float4 a, b, c, d; float4 arow[3]; WfMeta meta; };
struct __align__(128) WfVtx { float4 x_tu, ng_tv, wi_pdf, wl_ps, misc, mat; int4 ids; float4 pad; };
struct __align__(16) WfRay { float4 o_tmax, dir; };
static_assert(sizeof(WfPath) == 128 && sizeof(WfVtx) == 128, "one 128-byte record per path");

enum : unsigned {
    kFEmit = 1u, kFOutside = 2u, kFOk = 4u, kFTerminal = 8u, kFDelta = 16u, kFHit = 32u,
    kEvShift = 6, kNeeShift = 8
};

__device__ __forceinline__ void put_walk(WfPath* p, const Walk& w) {
    p->a = make_float4(w.o.x, w.o.y, w.o.z, w.prev_pdf);
    p->b = make_float4(w.d.x, w.d.y, w.d.z, __uint_as_float(w.sig));
    p->c = make_float4(w.xprev.x, w.xprev.y, w.xprev.z,
                       __int_as_float(w.v | (w.nv << 8) | ((w.prev_delta ? 1 : 0) << 16)));
    p->d = make_float4(w.d1.x, w.d1.y, w.d1.z, 0.0f);
}
__device__ __forceinline__ void get_walk(const WfPath* p, Walk& w) {
    const float4 a = p->a, b = p->b, c = p->c, d = p->d;
    w.o = {a.x, a.y, a.z}; w.prev_pdf = a.w;
    w.d = {b.x, b.y, b.z}; w.sig = __float_as_uint(b.w);
    w.xprev = {c.x, c.y, c.z};
    int bits = __float_as_int(c.w);
    w.v = bits & 0xff; w.nv = (bits >> 8) & 0xff; w.prev_delta = (bits >> 16) & 1;
    w.d1 = {d.x, d.y, d.z};
}

__device__ __forceinline__ void put_vertex(WfVtx* p, const VCtx& vc, const NeePending& ne, const Shade& sh) {
    WfVtx r;
    r.x_tu = make_float4(vc.x.x, vc.x.y, vc.x.z, vc.tu);
    r.ng_tv = make_float4(vc.ng.x, vc.ng.y, vc.ng.z, vc.tv);
    r.wi_pdf = make_float4(sh.wi.x, sh.wi.y, sh.wi.z, sh.pdf);
    r.wl_ps = make_float4(ne.wl.x, ne.wl.y, ne.wl.z, vc.pspec);
    r.misc = make_float4(ne.pl, ne.cx, vc.w_emit, vc.p_event);
    r.mat = make_float4(vc.alpha, vc.alb[0], vc.alb[1], vc.alb[2]);
    unsigned f = kFHit | (vc.emit ? kFEmit : 0u) | (vc.outside ? kFOutside : 0u) | (sh.ok ? kFOk : 0u) |
                 (sh.terminal ? kFTerminal : 0u) | (sh.delta ? kFDelta : 0u) | (sh.ev << kEvShift) |
                 ((unsigned)ne.state << kNeeShift);
    r.ids = make_int4(vc.prim, (vc.mat & 0xffff) | (ne.l << 16), vc.light, (int)f);
    r.pad = make_float4(0.f, 0.f, 0.f, 0.f);
    *p = r;
}
// (the ids first: a path whose ray missed reads 16 of the record's 112 bytes)
__device__ __forceinline__ bool get_vertex(const WfVtx* p, const Walk& w, VCtx& vc, NeePending& ne, Shade& sh) {
    WfVtx r;
    r.ids = p->ids;
    unsigned f = (unsigned)r.ids.w;
    if (!(f & kFHit)) return false;
    r.x_tu = p->x_tu; r.ng_tv = p->ng_tv; r.wi_pdf = p->wi_pdf; r.wl_ps = p->wl_ps; r.misc = p->misc; r.mat = p->mat;
    vc.x = {r.x_tu.x, r.x_tu.y, r.x_tu.z}; vc.tu = r.x_tu.w;
    vc.ng = {r.ng_tv.x, r.ng_tv.y, r.ng_tv.z}; vc.tv = r.ng_tv.w;
    vc.wo = -w.d;
    vc.n = dot(vc.ng, vc.wo) >= 0.0f ? vc.ng : -vc.ng;
    vc.prim = r.ids.x; vc.mat = r.ids.y & 0xffff; vc.light = r.ids.z;
    vc.emit = f & kFEmit; vc.outside = f & kFOutside;
    vc.w_emit = r.misc.z; vc.p_event = r.misc.w;
    vc.event = 0; vc.pdf = 1.0f; vc.nee = false; vc.scatter = false; vc.nee_light = -1; vc.nee_w = 0.0f;
    vc.wl = f3{0.f, 0.f, 0.f}; vc.wi = vc.wl;
    sh.wi = {r.wi_pdf.x, r.wi_pdf.y, r.wi_pdf.z}; sh.pdf = r.wi_pdf.w;
    sh.ok = f & kFOk; sh.terminal = f & kFTerminal; sh.delta = f & kFDelta; sh.ev = (f >> kEvShift) & 3u;
    ne.state = (int)((f >> kNeeShift) & 3u);
    ne.l = r.ids.y >> 16;
    ne.wl = {r.wl_ps.x, r.wl_ps.y, r.wl_ps.z}; vc.pspec = r.wl_ps.w;
    ne.pl = r.misc.x; ne.cx = r.misc.y;
    vc.alpha = r.mat.x; vc.alb[0] = r.mat.y; vc.alb[1] = r.mat.z; vc.alb[2] = r.mat.w;
    return true;
}

constexpr int kMissCode = (int)0x80000000;

struct WfState {
    WfPath* path;
    WfVtx* vtx;
    float4* hit;        // (t, b1, b2, BVH slot | -(sphere + 1) | kMissCode)
    WfRay* ray;         // shadow rays
    int* visible;
    float4* raw;        // raw Stokes per path, 3 per path
    float* cache;
    long long Q;
    int cap;
    __device__ __forceinline__ float* rec(int v, int q) const { return cache + ((long long)v * Q + q) * kWfCacheComps; }
};
// the code of a traversal's result: the BVH slot of a triangle, -(sphere + 1), or kMissCode
__device__ __forceinline__ int code_of(const DScene& S, bool hit, const HitRec& h) {
    return !hit ? kMissCode : h.prim < S.num_tris ? h.slot : -(h.prim - S.num_tris + 1);
}
// the hit of a code (not a miss)
__device__ __forceinline__ void decode_hit(const DScene& S, const float4& hv, HitRec& h) {
    const int code = __float_as_int(hv.w);
    h.t = hv.x; h.b1 = hv.y; h.b2 = hv.z;
    if (code >= 0) { h.slot = code; h.prim = __float_as_int(__ldg(&S.tris[3 * code].w)); }
    else { h.slot = -1; h.prim = S.num_tris + (-code - 1); }
}

struct WfLists {
    int* l0;      // live paths of the cache pass
    int* next0;
    int* shadow;
    // counts of this iteration: [0] cache-pass paths, [4] shadow rays, [8 + b] replay bin b;
    // nxt: the same for the next iteration ([0] and [8 + b] are appended to).  The two
    // 16-int halves of the count array alternate between iterations, and each iteration's
    // k_wf_extend zeroes the counts the iteration appends to.
    int* cur;
    int* nxt;
    // replayed paths binned by the material type of their vertex: bin b at bins + b * binQ
    // (this iteration) and nbins + b * binQ (the next one)
    int* bins;
    int* nbins;
    int binQ;
};

// A wave: pieces of one or more jobs (whole pixels each) laid out back to back in the wave's
// path slots.  Piece k holds pixels pix0 .. pix0 + npix - 1 of job `job`, its paths in slots
// q0 .. q0 + npix * spp - 1 and its pixels at wave-pixel index qpix0 onward.
struct WaveSeg { int job, pad; long long pix0, npix, q0, qpix0; };
struct WaveTable {
    WaveSeg seg[kMaxJobsPerLaunch];
    int nseg, depth;          // pieces; the largest max_depth among them
    long long nq, npix;       // paths and pixels of the wave
};
// the piece holding wave slot q (pieces are sorted by q0)
__device__ __forceinline__ int wave_piece_of_slot(const WaveTable& wt, long long q) {
    int lo = 0, hi = wt.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (wt.seg[mid].q0 <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int wave_piece_of_pixel(const WaveTable& wt, long long i) {
    int lo = 0, hi = wt.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (wt.seg[mid].qpix0 <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}
// starts the path of wave slot q: camera ray, path record, job-local path id
__device__ __forceinline__ void wave_start_path(const DScene& S, const JobTable& T, const WaveTable& wt, int q,
                                                WfState& W, Walk& w) {
    const WaveSeg& sg = wt.seg[wave_piece_of_slot(wt, q)];
    const DJob& J = T.job[sg.job];
    const unsigned long long pid = (unsigned long long)(sg.pix0 * J.spp + (q - sg.q0));
    walk_begin(S, J, pid, (long long)(pid / J.spp), w);
    put_walk(W.path + q, w);
    W.path[q].meta = WfMeta{(unsigned)pid, (unsigned)(pid >> 32), sg.job, 0};
}

// Replay bins: the material types with a replay kernel of their own (diffuse, rough
// conductor, rough dielectric, polarizer and retarder sheets), and one bin for everything
// else (smooth dielectrics, emitter hits, paths that left the scene).
constexpr int kBinOther = 7;
// the bin word of a cache slot whose ray left the scene: the replay of a path ends at the
// vertex before it, with no launch for the miss
constexpr int kBinMiss = 15;
constexpr unsigned kBinnedTypes = (1u << DPPT_MAT_DIFFUSE) | (1u << DPPT_MAT_CONDUCTOR_GGX) |
                                  (1u << DPPT_MAT_PLASTIC_GGX) | (1u << DPPT_MAT_POLARIZER_SHEET) |
                                  (1u << DPPT_MAT_RETARDER_SHEET);

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


// Appends path q to the next iteration's replay bin b.  Appends are warp-aggregated: the
// lanes of a warp going to the same bin take consecutive slots with one atomic.
__device__ __forceinline__ void bin_append(const WfLists& L, int b, int q) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, b);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(L.nxt + 8 + b, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    L.nbins[(long long)b * L.binQ + base + __popc(peers & ((1u << lane) - 1u))] = q;
}

// The cache record's visibility word (kWfVisComp) holds, as an int, the light sample's
// visibility in bit 0 and the vertex's replay bin above it: the material type when that
// type has a replay kernel of its own, kBinMiss when the ray left the scene, else kBinOther.
__device__ __forceinline__ int replay_bin(const DScene& S, int mat) {
    const int t = __ldg(&S.mats[mat].type);
    return (kBinnedTypes >> t) & 1u ? t : kBinOther;
}
__device__ __forceinline__ int replay_bin_of(const WfState& W, int q, int v) {
    return __float_as_int(W.rec(v, q)[kWfVisComp]) >> 1;
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
            float* rec = W.rec(v - 1, q);
            *reinterpret_cast<float4*>(rec + kWfHitComp) = hv;
            if (miss) rec[kWfVisComp] = __int_as_float(kBinMiss << 1);
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
            float* rec = W.rec(w.v - 1, q);
            const int code = code_of(S, hit, h);
            *reinterpret_cast<float4*>(rec + kWfHitComp) =
                hit ? make_float4(h.t, h.b1, h.b2, __int_as_float(code)) : make_float4(0.f, 0.f, 0.f, __int_as_float(code));
            if (!hit) rec[kWfVisComp] = __int_as_float(kBinMiss << 1);
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
        vis.C.base = W.cache; vis.C.Q = W.Q; vis.C.q = q; vis.C.cap = W.cap;
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
            const float* rec = W.rec(w.v - 1, q);
            const float4 hv = *reinterpret_cast<const float4*>(rec + kWfHitComp);
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
                cont = walk_finish(S, P, w, vc, ne, (__float_as_int(rec[kWfVisComp]) & 1) != 0, sh, vis);
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

size_t wavefront_bytes(long long Q, int cap) {
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
    b += align_up(sizeof(float) * kWfCacheComps * (size_t)cap * Q);
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
                          void* ws, long long Q, int cap, int block, unsigned* status, cudaStream_t st,
                          StageLog* log) {
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
#if !DPPT_WF_FUSE_SHADE
        tok = log->begin(kStageWfInit, st);
        k_wf_init<<<grid, block, 0, st>>>(S, T, wt, W, A);
        log->end(tok, st);
#endif
        for (int it = 0; it < passes * wt.depth; ++it) {
            // lists, counts and bins alternate between two buffers: the next ones of an
            // iteration are the live ones of the following iteration
            const WfLists& L = (it & 1) ? B : A;
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
                tok = log->begin(kStageWfShadow, st);
                k_wf_shadow<<<grid, block, tsm, st>>>(S, W, L, status);
                log->end(tok, st);
                tok = log->begin(kStageWfCache, st);
                if (mode == 0) {
                    if (nmaps) k_wf_finish<0, 0, true><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                    else k_wf_finish<0, 0, false><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                } else {
                    if (nmaps) k_wf_finish<1, 0, true><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                    else k_wf_finish<1, 0, false><<<fgrid, 128, 0, st>>>(S, P, G, T, W, L);
                }
                log->end(tok, st);
            }
            if (mode == 1 && it > 0) {
                tok = log->begin(kStageWfReplay, st);
                // one replay kernel per binned material type present, then the other bin
                const ReplayArgs ra{S, P, G, T, W, L, fgrid, smem, st, nmaps};
                if (types & (1u << DPPT_MAT_CONDUCTOR_GGX)) launch_replay_bin<DPPT_MAT_CONDUCTOR_GGX>(ra);
                if (types & (1u << DPPT_MAT_PLASTIC_GGX)) launch_replay_bin<DPPT_MAT_PLASTIC_GGX>(ra);
                if (types & (1u << DPPT_MAT_DIFFUSE)) launch_replay_bin<DPPT_MAT_DIFFUSE>(ra);
                if (types & (1u << DPPT_MAT_POLARIZER_SHEET)) launch_replay_bin<DPPT_MAT_POLARIZER_SHEET>(ra);
                if (types & (1u << DPPT_MAT_RETARDER_SHEET)) launch_replay_bin<DPPT_MAT_RETARDER_SHEET>(ra);
                if (nmaps) k_wf_finish<1, 1, true, -1, kBinOther><<<fgrid, 128, smem, st>>>(S, P, G, T, W, L);
                else k_wf_finish<1, 1, false, -1, kBinOther><<<fgrid, 128, smem, st>>>(S, P, G, T, W, L);
                log->end(tok, st);
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
