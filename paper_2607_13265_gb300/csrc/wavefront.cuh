// The wavefront schedule's path records, lists and wave tables, shared by the stage kernels
// (wavefront.cu) and the hybrid-replay cache and replay kernels (wf_hybrid.cu).
#pragma once

#include "trace.cuh"

namespace dppt {

struct __align__(16) WfMeta { unsigned lo, hi; int job, pni; };  // pid, job, phase | n << 8 | i << 16
// a path's state: walk (o, prev_pdf) (d, sig) (xprev, v | nv | delta) (d1, -), adjoint row
// (3 channels), bookkeeping
struct __align__(128) WfPath { float4 a, b, c, d; float4 arow[3]; WfMeta meta; };
struct __align__(128) WfVtx { float4 x_tu, ng_tv, wi_pdf, wl_ps, misc, mat; int4 ids; float4 pad; };
struct __align__(16) WfRay { float4 o_tmax, dir; };
static_assert(sizeof(WfPath) == 128 && sizeof(WfVtx) == 128, "one 128-byte record per path");
static_assert(kSweepRecFloats == 16 && kSweepHitComp == 12 && kSweepRecFloats + 1 <= kWfCacheComps,
              "the sweep's records (suffix, hit) and visibility plane fit in the cache's space");

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
    // where the traversal stores each vertex's hit for the replay: the cache record of
    // (vertex slot, path) is rec_floats floats, its hit at hit_comp and its bin word at
    // vis_comp, or in vis_plane[vertex slot][path] (36, 32, 31: the cache of the cached
    // replay; 16, 12, plane: the sweep schedule's records; 4, 0, -1: the hits of the hybrid
    // replay, which keeps no bin word)
    int rec_floats, hit_comp, vis_comp;
    int* vis_plane;
    __device__ __forceinline__ float* rec(int v, int q) const { return cache + ((long long)v * Q + q) * rec_floats; }
    __device__ __forceinline__ float* hit_rec(int v, int q) const { return rec(v, q); }
    __device__ __forceinline__ int vis_word(int v, int q) const {
        return vis_plane ? vis_plane[(long long)v * Q + q] : __float_as_int(rec(v, q)[vis_comp]);
    }
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

// Replay bins: every material type has a replay kernel of its own (compiled for that type
// only, so that it holds no other type's code and registers); bin kBinOther, replayed by the
// kernel for any type, is kept for types without one.
constexpr int kBinOther = 7;
// the bin word of a cache slot whose ray left the scene: the replay of a path ends at the
// vertex before it, with no launch for the miss
constexpr int kBinMiss = 15;
constexpr unsigned kBinnedTypes = (1u << DPPT_MAT_DIFFUSE) | (1u << DPPT_MAT_SMOOTH_DIELECTRIC) |
                                  (1u << DPPT_MAT_CONDUCTOR_GGX) | (1u << DPPT_MAT_PLASTIC_GGX) |
                                  (1u << DPPT_MAT_POLARIZER_SHEET) | (1u << DPPT_MAT_RETARDER_SHEET) |
                                  (1u << DPPT_MAT_EMITTER);
static_assert(DPPT_MAT_EMITTER < kBinOther, "a binned type's bin is its type");

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
__device__ __forceinline__ int replay_bin_of(const WfState& W, int q, int v) { return W.vis_word(v, q) >> 1; }

// The cache the forward sweep folds: E_v and W_v from the thread-local arrays, the suffixes
// into the wave's per-vertex records (components 0-11 of kSweepRecFloats), where the replay
// reads them.
template <int MAXD>
struct SweepCache {
    LocalCache<MAXD> loc;
    GlobalCache glob;
    __device__ __forceinline__ void get_w(int v, Compact<float>& W) const { loc.get_w(v, W); }
    __device__ __forceinline__ void get_e(int v, float e[12]) const { loc.get_e(v, e); }
    __device__ __forceinline__ void put_e(int v, const float e[12]) const { glob.put_e(v, e); }
};

// The adjoint's forward sweep in one kernel (schedule DPPT_SCHED_SWEEP), one thread per wave
// slot: the thread runs its path to the end as the megakernel does (closest hit, shading,
// light sample and shadow ray, E_v and the compact W_v in thread-local arrays) and keeps per
// vertex only what the replay reads back: the closest hit (kSweepHitComp of the 64-byte
// record), the light sample's visibility with the vertex's replay bin (W.vis_plane), and after
// the backward fold the suffix L_v (components 0-11; L_0 too, although the replay never reads
// it, and zeros beside a miss's hit, so that every written 32-byte sector is written whole:
// a partly written sector costs the memory a read of it).  It then stores the path's raw Stokes value and
// starts the replay: the adjoint row of its pixel, the path in the bin of its first vertex,
// and the walk as begun, which went to the path record before the walk.  The replay's
// iterations run as in the wavefront schedule.
template <int MAXD, bool NM, int MT = -1>
__global__ void __launch_bounds__(256, DPPT_MIN_BLOCKS_PRIMAL)
k_wf_sweep(const DScene S, const DParams P, const __grid_constant__ JobTable T, const __grid_constant__ WaveTable wt,
           WfState W, WfLists L, unsigned* status) {
    float4 cE[MAXD][3];
    float4 cW[MAXD][5];
    const long long qq = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (qq >= wt.nq) return;
    const int q = (int)qq;
    const WaveSeg& sg = wt.seg[wave_piece_of_slot(wt, q)];
    const DJob& J = T.job[sg.job];
    const unsigned long long pid = (unsigned long long)(sg.pix0 * J.spp + (q - sg.q0));
    Walk w;
    walk_begin(S, J, pid, (long long)(pid / J.spp), w);
    put_walk(W.path + q, w);      // the replay's start: the same walk, begun again
    PathVis<LocalCache<MAXD>, MT, NM> vis;
    vis.S = &S; vis.P = &P; vis.G = nullptr; vis.sgrad = nullptr;
    vis.C.cE = cE; vis.C.cW = cW;
    vis.n = 0; vis.i = 0; vis.phase = 0; vis.has_last = false; vis.adjoint = true;
    for (;;) {
        HitRec h;
        const bool hit = trace_closest<false>(S, w.o, w.d, h, status, nullptr);
        if (!hit) {
            float4* rec = reinterpret_cast<float4*>(W.rec(w.v - 1, q));
            rec[kSweepHitComp / 4 - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            rec[kSweepHitComp / 4] = make_float4(0.f, 0.f, 0.f, __int_as_float(kMissCode));
            W.vis_plane[(long long)(w.v - 1) * W.Q + q] = kBinMiss << 1;
            break;
        }
        reinterpret_cast<float4*>(W.rec(w.v - 1, q))[kSweepHitComp / 4] =
            make_float4(h.t, h.b1, h.b2, __int_as_float(code_of(S, true, h)));
        VCtx vc;
        NeePending ne;
        Shade sh;
        walk_shade<NM, MT>(S, P, J, pid, w, h, vc, ne, sh);
        bool visible = false;
        if (ne.state == 1) visible = !trace_any<false>(S, ne.o2, ne.dir, ne.tmax, status, nullptr);
        // stored before walk_finish, so that nothing of it stays live through the vertex's
        // evaluation (the thread-local cache writes no record)
        W.vis_plane[(long long)(w.v - 1) * W.Q + q] = replay_bin(S, vc.mat) << 1 | (visible ? 1 : 0);
        if (!walk_finish<MT>(S, P, w, vc, ne, visible, sh, vis)) break;
    }
    SweepCache<MAXD> C;
    C.loc = vis.C;
    C.glob.base = W.cache; C.glob.Q = W.Q; C.glob.q = q; C.glob.cap = W.cap; C.glob.stride = kSweepRecFloats;
    float L0[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) L0[k] = vis.has_last ? vis.lastE[k] : 0.0f;
    int top = vis.n - 1;
    if (vis.has_last) {
        if (top >= 1) C.put_e(top, L0);
        --top;
    }
    fold_cached(C, top, true, L0);
    if (vis.n > 0) C.put_e(0, L0);
    const Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
    const float inv = 1.0f / (float)J.spp;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
        rot_apply(Rc, v);
        W.raw[3 * (long long)q + c] = make_float4(v[0] * inv, v[1] * inv, v[2] * inv, v[3] * inv);
    }
    if (vis.n == 0) {
        if (J.sig) J.sig[pid] = fnv(w.sig, (unsigned)w.nv);
        return;
    }
    const long long pix = (long long)(pid / J.spp);
    const float* ds = J.dS + pix * 12;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float av[4] = {__ldg(ds + 4 * c) * inv, __ldg(ds + 4 * c + 1) * inv, __ldg(ds + 4 * c + 2) * inv,
                       __ldg(ds + 4 * c + 3) * inv};
        rot_apply_row(Rc, av);
        W.path[q].arow[c] = make_float4(av[0], av[1], av[2], av[3]);
    }
    W.path[q].meta = WfMeta{(unsigned)pid, (unsigned)(pid >> 32), sg.job, 1 | (vis.n << 8)};
    bin_append(L, replay_bin_of(W, q, 0), q);
}

// one translation unit per cache depth instantiates the forward-sweep kernels and their launcher
#define DPPT_SWEEP_BUCKET(B)                                                                                        \
    cudaError_t launch_wf_sweep_##B(bool nmaps, const DScene& S, const DParams& P, const JobTable& T,              \
                                    const WaveTable& wt, const WfState& W, const WfLists& L, int block,           \
                                    unsigned* status, cudaStream_t st) {                                          \
        const long long g = (wt.nq + block - 1) / block;                                                         \
        if (g <= 0) return cudaSuccess;                                                                          \
        if (nmaps) k_wf_sweep<B, true><<<(int)g, block, 0, st>>>(S, P, T, wt, W, L, status);                       \
        else if ((S.mat_types & ~kDiffuseDielectricTypes) == 0)                                                  \
            k_wf_sweep<B, false, type_mask_mt(kDiffuseDielectricTypes)><<<(int)g, block, 0, st>>>(S, P, T, wt, W, L, \
                                                                                                  status);       \
        else k_wf_sweep<B, false><<<(int)g, block, 0, st>>>(S, P, T, wt, W, L, status);                           \
        return cudaGetLastError();                                                                               \
    }                                                                                                            \
    /* the attributes and occupancy of the kernel without normal-map code (the same launch  */                  \
    /* bounds as the one with it)                                                           */                  \
    cudaError_t sweep_attributes_##B(cudaFuncAttributes* a) {                                                   \
        return cudaFuncGetAttributes(a, reinterpret_cast<const void*>(&k_wf_sweep<B, false>));                   \
    }                                                                                                            \
    int sweep_occupancy_##B(int block) {                                                                         \
        int nb = 0;                                                                                              \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void*>(&k_wf_sweep<B, false>), \
                                                          block, 0) != cudaSuccess)                              \
            return 0;                                                                                            \
        return nb;                                                                                               \
    }

#define DPPT_DECLARE_SWEEP(B)                                                                                       \
    cudaError_t launch_wf_sweep_##B(bool nmaps, const DScene& S, const DParams& P, const JobTable& T,              \
                                    const WaveTable& wt, const WfState& W, const WfLists& L, int block,           \
                                    unsigned* status, cudaStream_t st);
DPPT_DECLARE_SWEEP(4)
DPPT_DECLARE_SWEEP(8)
DPPT_DECLARE_SWEEP(16)
DPPT_DECLARE_SWEEP(32)
DPPT_DECLARE_SWEEP(64)
DPPT_DECLARE_SWEEP(128)
#undef DPPT_DECLARE_SWEEP

}  // namespace dppt

namespace dppt {

// The hybrid cached replay (Sec. 4.4) in the wavefront schedule: the traversal stores each
// vertex's hit (16 B, in WfState's cache with a 4-float stride) and the cache pass its light
// sample's visibility (a byte), instead of the 144-byte cached vertex; per path the hybrid
// visitor keeps its block data [nb][60], route bytes [rstride], look-ahead [K][31], the
// replay's running block throughput and emission [60] and the flags of recomputed blocks
// [fw], all in the workspace (layout: wavefront_bytes with K > 1).
struct HybWs {
    float* ck;
    unsigned char* route;
    float* blk;
    float* btr;
    unsigned* flags;
    unsigned char* vis;     // [vertex slot][Q]
    int nb, rstride, fw;
    float gamma, eps;
};
// the hybrid's cache pass (phase 0) or replay (phase 1) over this iteration's cache-pass list
// or replay list (replay bin kBinOther), for checkpoint interval K in {4, 8, 16}
cudaError_t launch_wf_hybrid(int phase, int K, const DScene& S, const DParams& P, const DGrads& G,
                             const JobTable& T, const WfState& W, const WfLists& L, const HybWs& H, int grid,
                             size_t smem, cudaStream_t st);

}  // namespace dppt
