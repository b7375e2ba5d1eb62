// Device code of the polarized path tracer (sm_103a), included by one
// translation unit per cache-depth bucket.
//
// k_trace<MAXD, MODE> is the path-tracing megakernel: one thread per path,
// blocks take chunks of consecutive paths (one chunk per block in the grid
// schedule, chunks pulled from an atomic counter in the persistent schedule),
// and the spp paths of a pixel are summed with warp shuffles.
//  * MODE 0 (primal, phase 1 of path replay backpropagation, Sec. 3.2): each
//    path caches its per-vertex emission E_i and compact transport factor W_i
//    in thread-local arrays and folds them backward into L[1]; the lane sums
//    the sensor-frame Stokes vectors of its pixel.
//  * MODE 1 (adjoint, phases 2+3 with cached suffix replay, Sec. 4.3, Fig. 2):
//    the same cache pass and backward fold L[i] = E_i + W_i L[i+1] (stored over
//    E_i), then the replay regenerates the same path -- same Philox counters
//    and the same machine code, because both passes run through the single
//    call site of walk_step -- and accumulates a^T dE_i + a^T dW_i L[i+1] with
//    dual numbers before a <- a^T W_i.  No Mueller matrix is inverted.
#pragma once

#include <cfloat>
#include <type_traits>

#include "device_math.cuh"
#include "internal.h"

// resident 256-thread blocks per SM the register allocation must allow
// (2 -> at most 128 registers per thread, 1 -> at most 255)
#ifndef DPPT_MIN_BLOCKS_PRIMAL
#define DPPT_MIN_BLOCKS_PRIMAL 2
#endif
#ifndef DPPT_MIN_BLOCKS_ADJOINT
#define DPPT_MIN_BLOCKS_ADJOINT 1
#endif

namespace dppt {

enum : unsigned { kStatusStackOverflow = 1u };

// ================================================================== traversal
struct HitRec { float t; int prim, slot; float b1, b2; };

// work units of one path, gathered only by the instrumented primal instance
struct WorkCount {
    unsigned vertices, rays, shadow_rays, nodes, shadow_nodes, tri_tests, shadow_tri_tests, sph_tests, shadow_sph_tests;
};

// three-operand minimum / maximum (PTX min.f32 / max.f32 with three sources, sm_100+);
// like fminf / fmaxf they return the other operands when one is NaN
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ void child_slabs(float4 n0, float4 n1, float4 n2, f3 inv, f3 oi, float tmax,
                                            float& tl, float& tr, bool& hl, bool& hr) {
    float lx0 = fmaf(n0.x, inv.x, -oi.x), lx1 = fmaf(n0.y, inv.x, -oi.x);
    float ly0 = fmaf(n0.z, inv.y, -oi.y), ly1 = fmaf(n0.w, inv.y, -oi.y);
    float lz0 = fmaf(n2.x, inv.z, -oi.z), lz1 = fmaf(n2.y, inv.z, -oi.z);
    float rx0 = fmaf(n1.x, inv.x, -oi.x), rx1 = fmaf(n1.y, inv.x, -oi.x);
    float ry0 = fmaf(n1.z, inv.y, -oi.y), ry1 = fmaf(n1.w, inv.y, -oi.y);
    float rz0 = fmaf(n2.z, inv.z, -oi.z), rz1 = fmaf(n2.w, inv.z, -oi.z);
    float ln = fmax3(fminf(lx0, lx1), fminf(ly0, ly1), fmaxf(fminf(lz0, lz1), 0.0f));
    float lf = fmin3(fmaxf(lx0, lx1), fmaxf(ly0, ly1), fminf(fmaxf(lz0, lz1), tmax));
    float rn = fmax3(fminf(rx0, rx1), fminf(ry0, ry1), fmaxf(fminf(rz0, rz1), 0.0f));
    float rf = fmin3(fmaxf(rx0, rx1), fmaxf(ry0, ry1), fminf(fmaxf(rz0, rz1), tmax));
    hl = ln <= lf; hr = rn <= rf; tl = ln; tr = rn;
}

// Moller-Trumbore with precomputed edges; returns t or -1
__device__ __forceinline__ float tri_test(const float4* tris, int i, f3 o, f3 d, float& b1, float& b2) {
    float4 a = __ldg(tris + 3 * i), e1v = __ldg(tris + 3 * i + 1), e2v = __ldg(tris + 3 * i + 2);
    f3 v0 = {a.x, a.y, a.z}, e1 = {e1v.x, e1v.y, e1v.z}, e2 = {e2v.x, e2v.y, e2v.z};
    f3 pv = cross(d, e2);
    float det = dot(e1, pv);
    if (det == 0.0f) return -1.0f;
    float inv = 1.0f / det;
    f3 tv = o - v0;
    float u = dot(tv, pv) * inv;
    if (u < 0.0f || u > 1.0f) return -1.0f;
    f3 qv = cross(tv, e1);
    float w = dot(d, qv) * inv;
    if (w < 0.0f || u + w > 1.0f) return -1.0f;
    b1 = u; b2 = w;
    return dot(e2, qv) * inv;
}

__device__ __forceinline__ float sphere_test(float4 s, f3 o, f3 d, float tmax) {
    f3 l = o - f3{s.x, s.y, s.z};
    float beta = dot(l, d);
    f3 f = l - d * beta;
    float disc = s.w * s.w - dot(f, f);
    if (disc < 0.0f) return -1.0f;
    float gam = dot(l, l) - s.w * s.w;
    float h = -beta - copysignf(sqrtf(disc), beta);
    if (h == 0.0f) return -1.0f;
    float ta = gam / h, tb = h;
    float t0 = fminf(ta, tb), t1 = fmaxf(ta, tb);
    if (t0 > 0.0f && t0 < tmax) return t0;
    if (t1 > 0.0f && t1 < tmax) return t1;
    return -1.0f;
}

// 1 / d with components of magnitude below 1e-20 replaced by +-1e-20 (finite slab distances)
__device__ __forceinline__ float safe_rcp(float x) { return 1.0f / (fabsf(x) > 1e-20f ? x : copysignf(1e-20f, x)); }
__device__ __forceinline__ f3 safe_inv(f3 d) { return {safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z)}; }

// BVH traversal in the while-while form with postponed leaves (Aila & Laine,
// "Understanding the efficiency of ray traversal on GPUs", HPG 2009): a lane
// descends inner nodes until it has found a leaf, keeps descending while other
// lanes of its warp have not, and the warp then tests leaves together.
constexpr int kTravDone = 0x7fffffff;   // stack sentinel: traversal finished

// Traversal stacks.  LocalStack keeps all kBvhStack entries in thread-local memory.
// SharedStack keeps the top kShStack entries in the block's shared memory -- entry j of
// thread t at sh[j * blockDim.x], sh pointing at the thread's column, so the lanes of a warp
// use consecutive banks -- and the deeper ones in thread-local memory; the wavefront's
// traversal kernels use it when DPPT_TRAV_SHARED_STACK > 0.  Measured on the icosphere
// workload, 16 or 8 shared entries made the fused extend + shade stage slower (5.22 vs 4.95
// ms per step: the shared memory takes L1 capacity from the node fetches), so it is off.
#ifndef DPPT_TRAV_SHARED_STACK
#define DPPT_TRAV_SHARED_STACK 0
#endif
constexpr int kShStack = DPPT_TRAV_SHARED_STACK > 0 ? DPPT_TRAV_SHARED_STACK : 1;
struct LocalStack {
    int s[kBvhStack];
    __device__ __forceinline__ void put(int i, int v) { s[i] = v; }
    __device__ __forceinline__ int get(int i) const { return s[i]; }
};
struct SharedStack {
    int* sh;
    int loc[kBvhStack - kShStack];
    __device__ __forceinline__ void put(int i, int v) {
        if (i < kShStack) sh[i * blockDim.x] = v;
        else loc[i - kShStack] = v;
    }
    __device__ __forceinline__ int get(int i) const { return i < kShStack ? sh[i * blockDim.x] : loc[i - kShStack]; }
};
// dynamic shared memory of a traversal kernel launched with `block` threads
inline size_t trav_stack_smem(int block) { return DPPT_TRAV_SHARED_STACK > 0 ? sizeof(int) * kShStack * (size_t)block : 0; }

template <class St>
__device__ __forceinline__ int trav_pop(const St& st, int& sp) { return sp > 0 ? st.get(--sp) : kTravDone; }

// Traversal state of one ray, kept in registers between rounds (the stack is the
// caller's thread-local array).  t: best hit so far (closest) or the ray's tmax (any);
// prim: closest primitive id so far, or 1 once an any-hit query has found a blocker.
struct Trav {
    f3 o, d, inv, oi;
    float t, b1, b2;
    int prim, slot, sp, ref;
    int nx, ny, nz;     // 4-wide nodes: float4 offsets of the near planes per axis (far = near ^ 1)
};

__device__ __forceinline__ void trav_begin(Trav& r, f3 o, f3 d, float t) {
    r.o = o; r.d = d;
    r.inv = safe_inv(d);
    r.oi = {o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z};
    r.nx = r.inv.x < 0.0f ? 1 : 0;
    r.ny = r.inv.y < 0.0f ? 3 : 2;
    r.nz = r.inv.z < 0.0f ? 5 : 4;
    r.t = t; r.b1 = r.b2 = 0.0f;
    r.prim = -1; r.slot = -1; r.sp = 0; r.ref = 0;
}

// One round of the while-while loop with postponed leaves: inner nodes until this lane
// (and, while it waits, every lane of the warp in the round) has a leaf, then the leaves,
// including further leaves met on the stack.  ANY: stop at the first hit in (0, t).
// Returns true when the ray's traversal is complete.
template <bool ANY, bool COUNT, class St>
__device__ __forceinline__ bool trav_round(const DScene& S, Trav& r, St& stack, unsigned* status, WorkCount* wc) {
    int leaf = kTravDone;
    while (r.ref >= 0 && r.ref != kTravDone) {
        const float4* nd = S.nodes + 4 * r.ref;
        float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        float tl, tr; bool hl, hr;
        if (COUNT) { if (ANY) wc->shadow_nodes++; else wc->nodes++; }
        child_slabs(n0, n1, n2, r.inv, r.oi, r.t, tl, tr, hl, hr);
        int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
        if (hl && hr) {
            int nr = cl, fr = cr;
            if (!ANY && tr < tl) { nr = cr; fr = cl; }
            if (r.sp >= kBvhStack) { atomicOr(status, kStatusStackOverflow); r.ref = kTravDone; return true; }
            stack.put(r.sp++, fr);
            r.ref = nr;
        } else if (hl) r.ref = cl;
        else if (hr) r.ref = cr;
        else r.ref = trav_pop(stack, r.sp);
        if (r.ref < 0 && leaf == kTravDone) { leaf = r.ref; r.ref = trav_pop(stack, r.sp); }
        if (!__any_sync(__activemask(), leaf == kTravDone)) break;
    }
    while (leaf != kTravDone) {
        unsigned v = ~(unsigned)leaf;
        int first = (int)(v & 0x1FFFFFFu), cnt = (int)(v >> 25);
        if (COUNT) { if (ANY) wc->shadow_tri_tests += cnt; else wc->tri_tests += cnt; }
        for (int i = first; i < first + cnt; ++i) {
            float b1, b2;
            float t = tri_test(S.tris, i, r.o, r.d, b1, b2);
            if (ANY) {
                if (t > 0.0f && t < r.t) { r.prim = 1; r.ref = kTravDone; return true; }
            } else if (t > 0.0f && t <= r.t) {
                int id = __float_as_int(__ldg(&S.tris[3 * i].w));
                if (t < r.t || id < r.prim) { r.t = t; r.prim = id; r.slot = i; r.b1 = b1; r.b2 = b2; }
            }
        }
        leaf = kTravDone;
        if (r.ref < 0) { leaf = r.ref; r.ref = trav_pop(stack, r.sp); }
    }
    return r.ref == kTravDone;
}

// One round over the 4-wide BVH, with the same while-while structure: a node's four
// child boxes are tested together, the nearest hit child is descended and the other hits
// are pushed far to near (for any-hit queries in node order).  The slab test reads each
// axis's near and far planes by the sign of the ray direction (Williams et al., "An
// efficient and robust ray-box intersection algorithm", 2005), so no min/max of the two
// plane distances is needed.  COUNT counts a node visit as two units of two child boxes,
// the unit of the binary tree.
__device__ __forceinline__ void cswap(float& ta, int& ra, float& tb, int& rb) {
    if (tb < ta) { float t = ta; ta = tb; tb = t; int r = ra; ra = rb; rb = r; }
}
template <bool ANY, bool COUNT, class St>
__device__ __forceinline__ bool trav4_round(const DScene& S, Trav& r, St& stack, unsigned* status, WorkCount* wc) {
    int leaf = kTravDone;
    while (r.ref >= 0 && r.ref != kTravDone) {
        const float4* nd = S.nodes4 + 8 * r.ref;
        const float4 nx = __ldg(nd + r.nx), fx = __ldg(nd + (r.nx ^ 1));
        const float4 ny = __ldg(nd + r.ny), fy = __ldg(nd + (r.ny ^ 1));
        const float4 nz = __ldg(nd + r.nz), fz = __ldg(nd + (r.nz ^ 1)), rf = __ldg(nd + 6);
        const int cnt = __float_as_int(__ldg(&nd[7].x));
        if (COUNT) { if (ANY) wc->shadow_nodes += 2; else wc->nodes += 2; }
        const float bnx[4] = {nx.x, nx.y, nx.z, nx.w}, bfx[4] = {fx.x, fx.y, fx.z, fx.w};
        const float bny[4] = {ny.x, ny.y, ny.z, ny.w}, bfy[4] = {fy.x, fy.y, fy.z, fy.w};
        const float bnz[4] = {nz.x, nz.y, nz.z, nz.w}, bfz[4] = {fz.x, fz.y, fz.z, fz.w};
        const int cr[4] = {__float_as_int(rf.x), __float_as_int(rf.y), __float_as_int(rf.z), __float_as_int(rf.w)};
        float t[4];
        int c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float x0 = fmaf(bnx[k], r.inv.x, -r.oi.x), x1 = fmaf(bfx[k], r.inv.x, -r.oi.x);
            const float y0 = fmaf(bny[k], r.inv.y, -r.oi.y), y1 = fmaf(bfy[k], r.inv.y, -r.oi.y);
            const float z0 = fmaf(bnz[k], r.inv.z, -r.oi.z), z1 = fmaf(bfz[k], r.inv.z, -r.oi.z);
            const float tn = fmax3(x0, y0, fmaxf(z0, 0.0f));
            const float tf = fmin3(x1, y1, fminf(z1, r.t));
            const bool hit = k < cnt && tn <= tf;
            t[k] = hit ? tn : INFINITY;
            c[k] = hit ? cr[k] : kTravDone;
        }
        if (!ANY) {
            // sorting network on (t, ref): nearest first
            cswap(t[0], c[0], t[1], c[1]);
            cswap(t[2], c[2], t[3], c[3]);
            cswap(t[0], c[0], t[2], c[2]);
            cswap(t[1], c[1], t[3], c[3]);
            cswap(t[1], c[1], t[2], c[2]);
        }
        int next = kTravDone;
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            if (c[k] == kTravDone) continue;
            if (next != kTravDone) {
                if (r.sp >= kBvhStack) { atomicOr(status, kStatusStackOverflow); r.ref = kTravDone; return true; }
                stack.put(r.sp++, next);
            }
            next = c[k];
        }
        r.ref = next != kTravDone ? next : trav_pop(stack, r.sp);
        if (r.ref < 0 && leaf == kTravDone) { leaf = r.ref; r.ref = trav_pop(stack, r.sp); }
        if (!__any_sync(__activemask(), leaf == kTravDone)) break;
    }
    while (leaf != kTravDone) {
        unsigned v = ~(unsigned)leaf;
        int first = (int)(v & 0x1FFFFFFu), cnt = (int)(v >> 25);
        if (COUNT) { if (ANY) wc->shadow_tri_tests += cnt; else wc->tri_tests += cnt; }
        for (int i = first; i < first + cnt; ++i) {
            float b1, b2;
            float tt = tri_test(S.tris, i, r.o, r.d, b1, b2);
            if (ANY) {
                if (tt > 0.0f && tt < r.t) { r.prim = 1; r.ref = kTravDone; return true; }
            } else if (tt > 0.0f && tt <= r.t) {
                int id = __float_as_int(__ldg(&S.tris[3 * i].w));
                if (tt < r.t || id < r.prim) { r.t = tt; r.prim = id; r.slot = i; r.b1 = b1; r.b2 = b2; }
            }
        }
        leaf = kTravDone;
        if (r.ref < 0) { leaf = r.ref; r.ref = trav_pop(stack, r.sp); }
    }
    return r.ref == kTravDone;
}

// the traversal of the build's BVH layout
template <bool ANY, bool COUNT, class St>
__device__ __forceinline__ bool trav_step(const DScene& S, Trav& r, St& stack, unsigned* status, WorkCount* wc) {
    if (DPPT_BVH4) return trav4_round<ANY, COUNT>(S, r, stack, status, wc);
    return trav_round<ANY, COUNT>(S, r, stack, status, wc);
}

// spheres after the triangles: ties in t go to the lower primitive id (triangles first)
__device__ __forceinline__ void trav_spheres_closest(const DScene& S, Trav& r) {
    for (int k = 0; k < S.num_spheres; ++k) {
        float t = sphere_test(__ldg(S.spheres + k), r.o, r.d, FLT_MAX);
        int id = S.num_tris + k;
        if (t > 0.0f && (t < r.t || (t == r.t && id < r.prim))) { r.t = t; r.prim = id; r.slot = -1; }
    }
}
__device__ __forceinline__ bool trav_spheres_any(const DScene& S, f3 o, f3 d, float tmax) {
    for (int k = 0; k < S.num_spheres; ++k) {
        float t = sphere_test(__ldg(S.spheres + k), o, d, tmax);
        if (t > 0.0f && t < tmax) return true;
    }
    return false;
}

// closest hit; ties in t go to the lower primitive id (triangles before spheres).  St: the
// traversal stack (LocalStack, or SharedStack in kernels that provide shared memory for it).
template <bool COUNT, class St>
__device__ bool trace_closest_with(const DScene& S, f3 o, f3 d, HitRec& h, unsigned* status, WorkCount* wc, St& stack) {
    if (COUNT) { wc->rays++; wc->sph_tests += S.num_spheres; }
    Trav r;
    trav_begin(r, o, d, FLT_MAX);
    if (S.num_tris > 0) {
        while (!trav_step<false, COUNT>(S, r, stack, status, wc)) {
        }
    }
    trav_spheres_closest(S, r);
    h.t = r.t; h.prim = r.prim; h.slot = r.slot; h.b1 = r.b1; h.b2 = r.b2;
    return h.prim >= 0;
}
template <bool COUNT>
__device__ bool trace_closest(const DScene& S, f3 o, f3 d, HitRec& h, unsigned* status, WorkCount* wc) {
    LocalStack stack;
    return trace_closest_with<COUNT>(S, o, d, h, status, wc, stack);
}

// any hit in (0, tmax)
template <bool COUNT, class St>
__device__ bool trace_any_with(const DScene& S, f3 o, f3 d, float tmax, unsigned* status, WorkCount* wc, St& stack) {
    if (COUNT) { wc->shadow_rays++; wc->shadow_sph_tests += S.num_spheres; }
    if (trav_spheres_any(S, o, d, tmax)) return true;
    if (S.num_tris == 0) return false;
    Trav r;
    trav_begin(r, o, d, tmax);
    while (!trav_step<true, COUNT>(S, r, stack, status, wc)) {
    }
    return r.prim >= 0;
}
template <bool COUNT>
__device__ bool trace_any(const DScene& S, f3 o, f3 d, float tmax, unsigned* status, WorkCount* wc) {
    LocalStack stack;
    return trace_any_with<COUNT>(S, o, d, tmax, status, wc, stack);
}

// ================================================================== textures
struct Taps { long long idx[4]; float w[4]; };
// a mod n in [0, n); texel coordinates are nearly always within one period of the range
__device__ __forceinline__ int wrapi(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    if (a < 0 && a >= -n) return a + n;
    if (a >= n && a < 2 * n) return a - n;
    int m = a % n;
    return m < 0 ? m + n : m;
}
__device__ __forceinline__ Taps tex_taps(const DTex& t, float u, float v) {
    float x = u * (float)t.w - 0.5f, y = v * (float)t.h - 0.5f;
    float fx0 = floorf(x), fy0 = floorf(y);
    float fx = x - fx0, fy = y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0;
    int xa = wrapi(x0, t.w), xb = wrapi(x0 + 1, t.w), ya = wrapi(y0, t.h), yb = wrapi(y0 + 1, t.h);
    Taps tp;
    tp.idx[0] = t.off + ((long long)ya * t.w + xa) * t.ch; tp.w[0] = (1.0f - fx) * (1.0f - fy);
    tp.idx[1] = t.off + ((long long)ya * t.w + xb) * t.ch; tp.w[1] = fx * (1.0f - fy);
    tp.idx[2] = t.off + ((long long)yb * t.w + xa) * t.ch; tp.w[2] = (1.0f - fx) * fy;
    tp.idx[3] = t.off + ((long long)yb * t.w + xb) * t.ch; tp.w[3] = fx * fy;
    return tp;
}
__device__ __forceinline__ float tex_value(const float* data, const Taps& tp, int c) {
    return __ldg(data + tp.idx[0] + c) * tp.w[0] + __ldg(data + tp.idx[1] + c) * tp.w[1] +
           __ldg(data + tp.idx[2] + c) * tp.w[2] + __ldg(data + tp.idx[3] + c) * tp.w[3];
}
__device__ __forceinline__ float tex_lookup(const DScene& S, const float* data, int tex, int c, float u, float v) {
    DTex t = S.tex[tex];
    Taps tp = tex_taps(t, u, v);
    return tex_value(data, tp, min(c, t.ch - 1));
}

// ================================================================== vertex context
// One vertex of a sampled path.  Sampling uses the (detached) parameter values;
// the Mueller values are evaluated from this record (float or dual numbers).
struct VCtx {
    f3 x, ng, n, wo, wl, wi;
    float tu, tv, w_emit, nee_w, pdf, p_event;
    float alpha, alb[3], pspec;   // material values at the vertex, looked up once
    int prim, mat, light, nee_light, event;
    bool emit, nee, scatter, outside;
};

__device__ __forceinline__ float ggx_pdf(float alpha, f3 n, f3 wo, f3 wi) {
    f3 h = normalize(wo + wi);
    float ch = dot(h, n), oh = dot(wo, h);
    if (ch <= 0.0f || oh <= 0.0f) return 0.0f;
    const f3 nh = cross(n, h);
    return ggx_D<float>(ch, dot(nh, nh), alpha) * ch / (4.0f * oh);
}
// Roughness, albedo (tint) and the rough dielectric's specular-lobe probability at the
// vertex: looked up once and reused by sampling, pdfs and the Mueller evaluation.
__device__ __forceinline__ void material_values(const DScene& S, const DParams& P, const DMat& m, VCtx& vc) {
    if (m.albedo_tex >= 0) {
        DTex t = S.tex[m.albedo_tex];
        Taps tp = tex_taps(t, vc.tu, vc.tv);
        for (int c = 0; c < 3; ++c) vc.alb[c] = tex_value(P.tex, tp, min(c, t.ch - 1));
    } else {
        vc.alb[0] = vc.alb[1] = vc.alb[2] = 1.0f;
    }
    vc.alpha = 0.0f;
    vc.pspec = 0.0f;
    if (m.type == DPPT_MAT_CONDUCTOR_GGX || m.type == DPPT_MAT_PLASTIC_GGX)
        vc.alpha = tex_lookup(S, P.tex, m.rough_tex, 0, vc.tu, vc.tv);
    if (m.type == DPPT_MAT_PLASTIC_GGX) {
        float eta = __ldg(P.ior + m.ior_index);
        float fs = fresnel_unpolarized(dot(vc.wo, vc.n), 1.0f, eta);
        float fd = (vc.alb[0] + vc.alb[1] + vc.alb[2]) / 3.0f;
        float tot = fs + fd;
        vc.pspec = tot > 0.0f ? fs / tot : 0.5f;
    }
}
__device__ __forceinline__ float bsdf_pdf(const DScene& S, const DParams& P, const DMat& m, const VCtx& vc, f3 wi) {
    float ci = dot(wi, vc.n);
    if (ci <= 0.0f) return 0.0f;
    if (m.type == DPPT_MAT_DIFFUSE) return ci * kInvPi;
    if (m.type == DPPT_MAT_CONDUCTOR_GGX) return ggx_pdf(vc.alpha, vc.n, vc.wo, wi);
    if (m.type == DPPT_MAT_PLASTIC_GGX)
        return vc.pspec * ggx_pdf(vc.alpha, vc.n, vc.wo, wi) + (1.0f - vc.pspec) * ci * kInvPi;
    return 0.0f;
}

__device__ __forceinline__ unsigned fnv(unsigned h, unsigned x) {
#pragma unroll
    for (int k = 0; k < 4; ++k) { h ^= (x >> (8 * k)) & 0xffu; h *= 16777619u; }
    return h;
}

__device__ __forceinline__ DLight load_light(const DScene& S, int l) { return S.lights[l]; }

// ================================================================== compact Mueller operators
// W = R(ro) . M . R(ri) per channel with M = [[A+D,B,0,0],[B,A,0,0],[0,0,C,S],[0,0,-S,C]]:
// every operator of the scene (depolarizer, Fresnel R/T, pBRDF lobes, polarizer,
// retarder) has this form in its own s/p or axis frame.
template <class T> struct Compact {
    Rot<T> ri, ro;
    T A[3], B[3], C[3], S[3], D[3];
};
template <class T> __device__ __forceinline__ void compact_zero(Compact<T>& W) {
    W.ri = {T(1.0f), T(0.0f)}; W.ro = {T(1.0f), T(0.0f)};
    for (int c = 0; c < 3; ++c) W.A[c] = W.B[c] = W.C[c] = W.S[c] = W.D[c] = T(0.0f);
}
// y = W_c x  (column)
template <class T, class V> __device__ __forceinline__ void compact_apply(const Compact<T>& W, int c, const V x[4], V y[4]) {
    V v[4] = {x[0], x[1], x[2], x[3]};
    rot_apply(W.ri, v);
    y[0] = (W.A[c] + W.D[c]) * v[0] + W.B[c] * v[1];
    y[1] = W.B[c] * v[0] + W.A[c] * v[1];
    y[2] = W.C[c] * v[2] + W.S[c] * v[3];
    y[3] = W.C[c] * v[3] - W.S[c] * v[2];
    rot_apply(W.ro, y);
}
// a^T <- a^T W_c  (row)
template <class V> __device__ __forceinline__ void compact_row(const Compact<float>& W, int c, V a[4]) {
    V u[4] = {a[0], a[1], a[2], a[3]};
    rot_apply_row(W.ro, u);
    a[0] = u[0] * (W.A[c] + W.D[c]) + u[1] * W.B[c];
    a[1] = u[0] * W.B[c] + u[1] * W.A[c];
    a[2] = u[2] * W.C[c] - u[3] * W.S[c];
    a[3] = u[2] * W.S[c] + u[3] * W.C[c];
    rot_apply_row(W.ri, a);
}
__device__ __forceinline__ Compact<float> compact_value(const Compact<D1>& W) {
    Compact<float> r;
    r.ri = {W.ri.c.v, W.ri.s.v}; r.ro = {W.ro.c.v, W.ro.s.v};
    for (int c = 0; c < 3; ++c) { r.A[c] = W.A[c].v; r.B[c] = W.B[c].v; r.C[c] = W.C[c].v; r.S[c] = W.S[c].v; r.D[c] = W.D[c].v; }
    return r;
}
__device__ __forceinline__ Compact<float> compact_value(const Compact<D2>& W) {
    Compact<float> r;
    r.ri = {W.ri.c.v, W.ri.s.v}; r.ro = {W.ro.c.v, W.ro.s.v};
    for (int c = 0; c < 3; ++c) { r.A[c] = W.A[c].v; r.B[c] = W.B[c].v; r.C[c] = W.C[c].v; r.S[c] = W.S[c].v; r.D[c] = W.D[c].v; }
    return r;
}
__device__ __forceinline__ Compact<float> compact_value(const Compact<D3>& W) {
    Compact<float> r;
    r.ri = {W.ri.c.v, W.ri.s.v}; r.ro = {W.ro.c.v, W.ro.s.v};
    for (int c = 0; c < 3; ++c) { r.A[c] = W.A[c].v; r.B[c] = W.B[c].v; r.C[c] = W.C[c].v; r.S[c] = W.S[c].v; r.D[c] = W.D[c].v; }
    return r;
}

template <class T> __device__ __forceinline__ T seeded(float v, int slot) {
    return T(v);
}
template <> __device__ __forceinline__ D3 seeded<D3>(float v, int slot) {
    return D3(v, slot == 0 ? 1.0f : 0.0f, slot == 1 ? 1.0f : 0.0f, slot == 2 ? 1.0f : 0.0f);
}
// D1 carries slot 2 (the channel albedo) alone, D2 slots 0 and 2
template <> __device__ __forceinline__ D1 seeded<D1>(float v, int slot) { return D1(v, slot == 2 ? 1.0f : 0.0f); }
template <> __device__ __forceinline__ D2 seeded<D2>(float v, int slot) {
    return D2(v, slot == 0 ? 1.0f : 0.0f, slot == 2 ? 1.0f : 0.0f);
}
// the derivatives of the three slots (roughness or sheet angle, index of refraction, albedo)
__device__ __forceinline__ float dslot0(const D3& x) { return x.d0; }
__device__ __forceinline__ float dslot1(const D3& x) { return x.d1; }
__device__ __forceinline__ float dslot2(const D3& x) { return x.d2; }
__device__ __forceinline__ float dslot0(const D1&) { return 0.0f; }
__device__ __forceinline__ float dslot1(const D1&) { return 0.0f; }
__device__ __forceinline__ float dslot2(const D1& x) { return x.d; }
__device__ __forceinline__ float dslot0(const D2& x) { return x.d0; }
__device__ __forceinline__ float dslot1(const D2&) { return 0.0f; }
__device__ __forceinline__ float dslot2(const D2& x) { return x.d2; }

// s axis of a reflection/refraction: normal to the plane of (a, b), or any
// axis normal to a when the plane degenerates
__device__ __forceinline__ f3 s_axis(f3 a, f3 b) {
    f3 sx = cross(a, b);
    float sl = len(sx);
    return sl > 1e-12f ? sx * (1.0f / sl) : onb_t1(a);
}

// Normal maps: the shading normal normalize(n.x T + n.y B + n.z N) of a triangle vertex,
// n = 2 c - 1 from the material's tangent-space map (bilinear), N the geometric normal on
// the side of wo, T the triangle's dP/du made normal to N and unit, B = N x T.  For T = D3
// the three components of n are the dual-number slots (a normal-mapped material's texel
// derivatives replace its albedo / roughness / index slots).  Returns false, leaving n,
// when the vertex has no usable normal map.
__device__ __forceinline__ bool nmap_frame(const DScene& S, const DMat& m, const VCtx& vc, f3& N, f3& Tg, f3& B) {
    if (m.normal_tex < 0 || vc.prim >= S.num_tris || !S.tri_tan) return false;
    N = dot(vc.ng, vc.wo) >= 0.0f ? vc.ng : -vc.ng;
    f3 t = ld3(S.tri_tan + 3 * (long long)vc.prim);
    t = t - N * dot(N, t);
    const float tl = len(t);
    if (!(tl > 1e-12f)) return false;
    Tg = t * (1.0f / tl);
    B = cross(N, Tg);
    return true;
}
template <class T>
__device__ __forceinline__ bool shading_normal(const DScene& S, const DParams& P, const DMat& m, const VCtx& vc,
                                               T n[3]) {
    f3 N, Tg, B;
    if (!nmap_frame(S, m, vc, N, Tg, B)) return false;
    const Taps tp = tex_taps(S.tex[m.normal_tex], vc.tu, vc.tv);
    T a[3];
    for (int c = 0; c < 3; ++c) a[c] = seeded<T>(2.0f * tex_value(P.tex, tp, c) - 1.0f, c);
    T x = a[0] * Tg.x + a[1] * B.x + a[2] * N.x;
    T y = a[0] * Tg.y + a[1] * B.y + a[2] * N.y;
    T z = a[0] * Tg.z + a[1] * B.z + a[2] * N.z;
    T l = tsqrt(x * x + y * y + z * z);
    n[0] = x / l; n[1] = y / l; n[2] = z / l;
    return true;
}
// the vertex's detached shading normal into vc.n (no-op without a normal map)
__device__ __forceinline__ void apply_normal_map(const DScene& S, const DParams& P, VCtx& vc) {
    const DMat m = S.mats[vc.mat];
    float n[3];
    if (m.normal_tex >= 0 && shading_normal<float>(S, P, m, vc, n)) vc.n = f3{n[0], n[1], n[2]};
}

// pBRDF value f(wo, wi) without the cosine, as a compact operator.  NM: the shading normal
// nT carries derivatives (normal map); the material's own parameters are then constants.
template <class T, bool NM = false>
__device__ __forceinline__ void bsdf_compact(const DScene& S, const DParams& P, const DMat& m, const VCtx& vc, f3 wi,
                                             Compact<T>& f, const T* nT = nullptr) {
    using C = typename std::conditional<NM, T, float>::type;
    compact_zero(f);
    C ci, co;
    if constexpr (NM) {
        ci = nT[0] * wi.x + nT[1] * wi.y + nT[2] * wi.z;
        co = nT[0] * vc.wo.x + nT[1] * vc.wo.y + nT[2] * vc.wo.z;
    } else {
        ci = dot(wi, vc.n);
        co = dot(vc.wo, vc.n);
    }
    if (val(ci) <= 0.0f || val(co) <= 0.0f) return;
    T alb[3];
    if (m.albedo_tex >= 0) {
        for (int c = 0; c < 3; ++c) alb[c] = seeded<T>(vc.alb[c], NM ? -1 : 2);
    } else {
        for (int c = 0; c < 3; ++c) alb[c] = T(1.0f);
    }
    if (m.type == DPPT_MAT_DIFFUSE) {
        for (int c = 0; c < 3; ++c) f.D[c] = alb[c] * kInvPi;
        return;
    }
    f3 h = normalize(vc.wo + wi);
    C ch, sh2;   // cosine and squared sine (|n x h|^2) of the half vector's angle to the normal
    if constexpr (NM) {
        ch = nT[0] * h.x + nT[1] * h.y + nT[2] * h.z;
        const C cx = nT[1] * h.z - nT[2] * h.y, cy = nT[2] * h.x - nT[0] * h.z, cz = nT[0] * h.y - nT[1] * h.x;
        sh2 = cx * cx + cy * cy + cz * cz;
    } else {
        ch = dot(h, vc.n);
        const f3 nh = cross(vc.n, h);
        sh2 = dot(nh, nh);
    }
    const float oh = dot(vc.wo, h), ih = dot(wi, h);
    T al = seeded<T>(vc.alpha, NM ? -1 : 0);
    T k = ggx_D<T, C>(ch, sh2, al) * ggx_G1<T, C>(co, oh, al) * ggx_G1<T, C>(ci, ih, al) / (co * ci * 4.0f);
    ABCS<T> F;
    if (m.type == DPPT_MAT_CONDUCTOR_GGX) {
        ABCS<float> Ff = fresnel_reflect<float>(ih, 1.0f, Cx<float>{m.eta_re, m.eta_im});
        F = {T(Ff.A), T(Ff.B), T(Ff.C), T(Ff.S)};
    } else {
        F = fresnel_reflect_real<T>(ih, T(1.0f), seeded<T>(__ldg(P.ior + m.ior_index), NM ? -1 : 1));
    }
    f3 sax = s_axis(vc.wo, h);
    Rot<float> ri = rot_between(-wi, onb_t1(-wi), sax);
    Rot<float> ro = rot_between(vc.wo, sax, onb_t1(vc.wo));
    f.ri = {T(ri.c), T(ri.s)}; f.ro = {T(ro.c), T(ro.s)};
    for (int c = 0; c < 3; ++c) {
        T kc = m.type == DPPT_MAT_CONDUCTOR_GGX ? k * alb[c] : k;
        f.A[c] = F.A * kc; f.B[c] = F.B * kc; f.C[c] = F.C * kc; f.S[c] = F.S * kc;
        if (m.type == DPPT_MAT_PLASTIC_GGX) f.D[c] = alb[c] * kInvPi;
    }
}

template <class T, class U> __device__ __forceinline__ void compact_scale(Compact<T>& W, U s) {
    for (int c = 0; c < 3; ++c) { W.A[c] = W.A[c] * s; W.B[c] = W.B[c] * s; W.C[c] = W.C[c] * s; W.S[c] = W.S[c] * s; W.D[c] = W.D[c] * s; }
}

// Emitted Stokes of light l arriving along propagation p, rotated from the
// emitter frame (x = e1 projected) into the canonical frame of p.
__device__ __forceinline__ Rot<float> emitter_rot(const DLight& L, f3 p) {
    f3 e1 = ld3(L.e1);
    f3 xe = e1 - p * dot(e1, p);
    return rot_between(p, xe, onb_t1(p));
}

// Material-type specializations of a kernel: MT >= 0 is one type, -1 any type, and
// type_mask_mt(mask) a set of types (kernels for scenes whose materials all have a type of
// the set; the host chooses them from DScene::mat_types).
constexpr int type_mask_mt(unsigned mask) { return -2 - (int)mask; }
// diffuse surfaces, smooth dielectrics and emitters: a Cornell box
constexpr unsigned kDiffuseDielectricTypes =
    (1u << DPPT_MAT_DIFFUSE) | (1u << DPPT_MAT_SMOOTH_DIELECTRIC) | (1u << DPPT_MAT_EMITTER);
// The type t written as a choice among the types of TM: every comparison of it with a type
// outside TM then folds to false at compile time.
template <unsigned TM>
__device__ __forceinline__ int typed_as(int t) {
    constexpr int hi = 31 - __builtin_clz(TM);
    int r = hi;
#pragma unroll
    for (int k = 0; k < hi; ++k)
        if ((TM >> k) & 1u) r = t == k ? k : r;
    return r;
}
// The material of a vertex; MT >= 0 states its type at compile time (kernels specialized
// to one material type) and MT < -1 the set its type belongs to, so that the other types'
// code folds away.
template <int MT>
__device__ __forceinline__ DMat load_mat(const DScene& S, int mat) {
    DMat m = S.mats[mat];
    if constexpr (MT >= 0) m.type = MT;
    else if constexpr (MT < -1) m.type = typed_as<(unsigned)(-MT - 2)>(m.type);
    return m;
}

// E_v (per channel, float) and W_v (compact, T) for one vertex.  NM = false compiles the
// normal-map path out (kernels launched for scenes without normal maps).  With dual numbers
// the three slots carry the material's own parameters (roughness or sheet angle, index of
// refraction, channel albedo) and the shading normal is a constant; NSLOTS instead makes
// them the components of a normal-mapped vertex's map value n, the material's parameters
// then being constants (replay_vjp runs both evaluations at such a vertex).
template <class T, int MT = -1, bool NM = true, bool NSLOTS = false>
__device__ void eval_vertex(const DScene& S, const DParams& P, const VCtx& vc, float E[3][4], Compact<T>& W,
                            Compact<T>* fnee) {
    const DMat m = load_mat<MT>(S, vc.mat);
    for (int c = 0; c < 3; ++c) E[c][0] = E[c][1] = E[c][2] = E[c][3] = 0.0f;
    if (vc.emit) {
        DLight L = load_light(S, vc.light);
        Rot<float> R = emitter_rot(L, vc.wo);
        for (int c = 0; c < 3; ++c) {
            const float* le = P.le + 12 * vc.light + 4 * c;
            float v[4] = {__ldg(le), __ldg(le + 1), __ldg(le + 2), __ldg(le + 3)};
            rot_apply(R, v);
            for (int k = 0; k < 4; ++k) E[c][k] = v[k] * vc.w_emit;
        }
    }
    if (m.emission > 0.0f)
        for (int c = 0; c < 3; ++c) E[c][0] += m.emission;
    // a normal map's shading normal with derivatives (the normal-slot evaluation only:
    // detached values are already in vc.n)
    T nT[3];
    bool nm = false;
    if constexpr (NM && NSLOTS && sizeof(T) != sizeof(float))
        if (m.normal_tex >= 0) nm = shading_normal<T>(S, P, m, vc, nT);
    if (vc.nee) {
        DLight L = load_light(S, vc.nee_light);
        Rot<float> R = emitter_rot(L, -vc.wl);
        Compact<T> f;
        if constexpr (NM && NSLOTS) {
            if (nm) {
                // nee_w holds the cosine with the detached shading normal: the live one replaces it
                bsdf_compact<T, true>(S, P, m, vc, vc.wl, f, nT);
                compact_scale(f, (nT[0] * vc.wl.x + nT[1] * vc.wl.y + nT[2] * vc.wl.z) * (1.0f / dot(vc.n, vc.wl)));
            } else {
                bsdf_compact<T>(S, P, m, vc, vc.wl, f);
            }
        } else {
            bsdf_compact<T>(S, P, m, vc, vc.wl, f);
        }
        Compact<float> fv;
        if constexpr (std::is_same<T, float>::value) fv = f;
        else fv = compact_value(f);
        for (int c = 0; c < 3; ++c) {
            const float* le = P.le + 12 * vc.nee_light + 4 * c;
            float v[4] = {__ldg(le), __ldg(le + 1), __ldg(le + 2), __ldg(le + 3)};
            rot_apply(R, v);
            float y[4];
            compact_apply(fv, c, v, y);
            for (int k = 0; k < 4; ++k) E[c][k] += y[k] * vc.nee_w;
        }
        if (fnee) *fnee = f;
    }
    compact_zero(W);
    if (!vc.scatter) return;
    f3 wi = vc.wi;
    if (m.type == DPPT_MAT_DIFFUSE || m.type == DPPT_MAT_CONDUCTOR_GGX || m.type == DPPT_MAT_PLASTIC_GGX) {
        if constexpr (NM && NSLOTS) {
            if (nm) {
                bsdf_compact<T, true>(S, P, m, vc, wi, W, nT);
                compact_scale(W, (nT[0] * wi.x + nT[1] * wi.y + nT[2] * wi.z) * (1.0f / vc.pdf));
            } else {
                bsdf_compact<T>(S, P, m, vc, wi, W);
                compact_scale(W, dot(wi, vc.n) / vc.pdf);
            }
        } else {
            bsdf_compact<T>(S, P, m, vc, wi, W);
            compact_scale(W, dot(wi, vc.n) / vc.pdf);
        }
    } else if (m.type == DPPT_MAT_SMOOTH_DIELECTRIC) {
        T eta = seeded<T>(__ldg(P.ior + m.ior_index), 1);
        T eo = vc.outside ? T(1.0f) : eta, et = vc.outside ? eta : T(1.0f);
        float c = dot(vc.wo, vc.n);
        f3 sax = s_axis(vc.wo, vc.n);
        Rot<float> ri = rot_between(-wi, onb_t1(-wi), sax);
        Rot<float> ro = rot_between(vc.wo, sax, onb_t1(vc.wo));
        ABCS<T> F;
        T sc;
        if (vc.event == 1) {
            F = fresnel_reflect_real<T>(c, eo, et);
            sc = T(1.0f / vc.p_event);
        } else {
            float ci = fabsf(dot(wi, vc.n));
            F = fresnel_transmit<T>(ci, et, eo);
            T q = eo / et;
            sc = q * q * (1.0f / vc.p_event);
        }
        W.ri = {T(ri.c), T(ri.s)}; W.ro = {T(ro.c), T(ro.s)};
        for (int cc = 0; cc < 3; ++cc) { W.A[cc] = F.A * sc; W.B[cc] = F.B * sc; W.C[cc] = F.C * sc; W.S[cc] = F.S * sc; }
    } else if (m.type == DPPT_MAT_POLARIZER_SHEET || m.type == DPPT_MAT_RETARDER_SHEET) {
        f3 p = vc.wo;
        T th = seeded<T>(__ldg(P.sheet + m.sheet_index), 0);
        T ct = tcos(th), st = tsin(th);
        T t[3] = {ct * m.t1[0] + st * m.t2[0], ct * m.t1[1] + st * m.t2[1], ct * m.t1[2] + st * m.t2[2]};
        T tp = t[0] * p.x + t[1] * p.y + t[2] * p.z;
        T xf[3] = {t[0] - tp * p.x, t[1] - tp * p.y, t[2] - tp * p.z};
        W.ri = rot_to_param<T>(p, onb_t1(p), xf);
        W.ro = rot_from_param<T>(p, xf, onb_t1(p));
        float A, B, C, Sv;
        if (m.type == DPPT_MAT_POLARIZER_SHEET) { A = 0.5f; B = 0.5f; C = 0.0f; Sv = 0.0f; }
        else { A = 1.0f; B = 0.0f; sincosf(m.retard, &Sv, &C); }
        for (int cc = 0; cc < 3; ++cc) { W.A[cc] = T(A); W.B[cc] = T(B); W.C[cc] = T(C); W.S[cc] = T(Sv); }
    }
}

// ================================================================== path walk
__device__ __forceinline__ f3 camera_dir(const DCam& c, int W, int H, int px, int py, float ju, float jv) {
    float aspect = (float)W / (float)H;
    float sx = (2.0f * ((float)px + ju) / (float)W - 1.0f) * c.tanh * aspect;
    float sy = (1.0f - 2.0f * ((float)py + jv) / (float)H) * c.tanh;
    return normalize(ld3(c.fwd) + ld3(c.right) * sx + ld3(c.up) * sy);
}
// rotation from the frame of light arriving at the camera along -d1 into the
// sensor frame (x = camera right projected normal to the ray)
__device__ __forceinline__ Rot<float> camera_rot(const DCam& c, f3 d1) {
    f3 p = -d1;
    f3 xr = ld3(c.right);
    f3 xs = xr - p * dot(xr, p);
    return rot_between(p, onb_t1(p), xs);
}

// State of the path a lane is tracing (sampling uses the detached parameters).
struct Walk {
    f3 o, d, xprev, d1;
    float prev_pdf;
    unsigned sig;
    int v, nv;
    bool prev_delta;
};

__device__ __forceinline__ void walk_begin(const DScene& S, const DJob& J, unsigned long long pid, long long pix,
                                           Walk& w) {
    const DCam& cam = S.cams[J.cam];
    U8 u0 = draw8(J.k0, J.k1, pid, 0u);
    w.d = camera_dir(cam, J.W, J.H, (int)(pix % J.W), (int)(pix / J.W), u0.u[0], u0.u[1]);
    w.d1 = w.d;
    w.o = ld3(cam.org);
    w.xprev = w.o;
    w.prev_delta = true;
    w.prev_pdf = 0.0f;
    w.sig = 2166136261u;
    w.v = 1;
    w.nv = 0;
}

// A vertex is produced in three steps so that the wavefront schedule can run
// them as separate kernels: walk_shade (given the closest hit: surface data,
// emission MIS weight, light sample and BSDF sample), the shadow ray of the
// light sample, and walk_finish (next-event weight, signature, per-vertex
// action, next ray).  walk_step chains them for the megakernel.
struct NeePending {
    f3 o2, dir, wl;
    float tmax, pl, cx;   // pl: solid-angle pdf of the light sample
    int l;
    int state;   // 2: no light sample at this vertex, 0: sample facing away, 1: shadow ray pending
};
struct Shade {
    f3 wi;
    float pdf;
    unsigned ev;
    bool ok, terminal, delta;
};

template <bool NM = true, int MT = -1>
__device__ __forceinline__ void walk_shade(const DScene& S, const DParams& P, const DJob& J, unsigned long long pid,
                                           const Walk& w, const HitRec& h, VCtx& vc, NeePending& ne, Shade& sh) {
    const int nL = S.num_lights;
    vc.prim = h.prim;
    vc.x = w.o + w.d * h.t;
    vc.wo = -w.d;
    vc.emit = vc.nee = vc.scatter = false;
    vc.event = 0; vc.w_emit = 0.0f; vc.nee_w = 0.0f; vc.pdf = 1.0f; vc.p_event = 1.0f;
    vc.outside = true; vc.nee_light = -1; vc.wl = f3{0.f, 0.f, 0.f}; vc.wi = vc.wl;
    if (h.prim < S.num_tris) {
        int f = h.prim;
        float4 e1v = __ldg(S.tris + 3 * h.slot + 1), e2v = __ldg(S.tris + 3 * h.slot + 2);
        vc.ng = normalize(cross(f3{e1v.x, e1v.y, e1v.z}, f3{e2v.x, e2v.y, e2v.z}));
        vc.mat = __ldg(S.tri_mat + f);
        vc.light = __ldg(S.tri_light + f);
        const float* uv = S.tri_uv + 6 * (long long)f;
        float w0 = 1.0f - h.b1 - h.b2;
        vc.tu = w0 * __ldg(uv) + h.b1 * __ldg(uv + 2) + h.b2 * __ldg(uv + 4);
        vc.tv = w0 * __ldg(uv + 1) + h.b1 * __ldg(uv + 3) + h.b2 * __ldg(uv + 5);
    } else {
        int k = h.prim - S.num_tris;
        float4 sp = __ldg(S.spheres + k);
        vc.ng = (vc.x - f3{sp.x, sp.y, sp.z}) * (1.0f / sp.w);
        vc.mat = __ldg(S.sph_mat + k);
        vc.tu = atan2f(vc.ng.z, vc.ng.x) * (0.5f * kInvPi) + 0.5f;
        vc.tv = acosf(fmaxf(-1.0f, fminf(1.0f, vc.ng.y))) * kInvPi;
        vc.light = -1;
    }
    vc.n = dot(vc.ng, vc.wo) >= 0.0f ? vc.ng : -vc.ng;
    const f3 ngo = vc.n;   // geometric normal on the side of wo
    const DMat m = load_mat<MT>(S, vc.mat);
    if (NM && m.normal_tex >= 0) apply_normal_map(S, P, vc);
    if (vc.light >= 0) {
        DLight L = load_light(S, vc.light);
        float cl = dot(ld3(L.n), vc.wo);
        if (cl > 0.0f) {
            vc.emit = true;
            if (w.prev_delta) vc.w_emit = 1.0f;
            else {
                f3 dx = vc.x - w.xprev;
                float pl = dot(dx, dx) / (cl * L.area * (float)nL);
                vc.w_emit = w.prev_pdf * w.prev_pdf / (w.prev_pdf * w.prev_pdf + pl * pl);
            }
        }
    }
    sh.ev = 0u;
    sh.ok = false;
    sh.pdf = 1.0f;
    sh.wi = f3{0.f, 0.f, 0.f};
    ne.state = 2;
    sh.terminal = m.type == DPPT_MAT_EMITTER || w.v == J.depth;
    sh.delta = m.type == DPPT_MAT_SMOOTH_DIELECTRIC || m.type == DPPT_MAT_POLARIZER_SHEET ||
               m.type == DPPT_MAT_RETARDER_SHEET;
    if (sh.terminal) return;
    material_values(S, P, m, vc);
    U8 U = draw8(J.k0, J.k1, pid, (unsigned)w.v);
    if (!sh.delta && nL > 0) {
        int l = min((int)(U.u[4] * (float)nL), nL - 1);
        DLight L = load_light(S, l);
        f3 y = ld3(L.o) + ld3(L.e1) * U.u[5] + ld3(L.e2) * U.u[6];
        f3 dv = y - vc.x;
        float dist2 = dot(dv, dv), dist = sqrtf(dist2);
        f3 wl = dv * (1.0f / dist);
        float cl = -dot(ld3(L.n), wl), cx = dot(vc.n, wl);
        ne.state = 0;
        if (cl > 0.0f && cx > 0.0f && dot(ngo, wl) > 0.0f) {
            f3 o2 = vc.x + ngo * S.eps;
            f3 dd = y - o2;
            float dl = len(dd);
            ne.o2 = o2;
            ne.dir = dd * (1.0f / dl);
            ne.tmax = dl * (1.0f - 1e-4f);
            ne.wl = wl;
            ne.pl = dist2 / (cl * L.area * (float)nL);
            ne.cx = cx;
            ne.l = l;
            ne.state = 1;
        }
    }
    bool ok = true;
    f3 wi = {0.f, 0.f, 0.f};
    if (m.type == DPPT_MAT_DIFFUSE || m.type == DPPT_MAT_PLASTIC_GGX || m.type == DPPT_MAT_CONDUCTOR_GGX) {
        bool spec = m.type == DPPT_MAT_CONDUCTOR_GGX;
        if (m.type == DPPT_MAT_PLASTIC_GGX) { spec = U.u[0] < vc.pspec; sh.ev = spec ? 1u : 2u; }
        f3 t1 = onb_t1(vc.n), t2 = onb_t2(vc.n);
        if (!spec) {
            float r = sqrtf(U.u[1]), sph, cph;
            sincosf(2.0f * kPi * U.u[2], &sph, &cph);
            wi = t1 * (r * cph) + t2 * (r * sph) + vc.n * sqrtf(fmaxf(0.0f, 1.0f - U.u[1]));
        } else {
            const float al = vc.alpha;
            float tan2 = al * al * U.u[1] / (1.0f - U.u[1]);
            float ch = 1.0f / sqrtf(1.0f + tan2);
            float shv = sqrtf(tan2) * ch;     // sin = tan cos: no cancellation near the normal
            float sph, cph;
            sincosf(2.0f * kPi * U.u[2], &sph, &cph);
            f3 hv = t1 * (shv * cph) + t2 * (shv * sph) + vc.n * ch;
            float oh = dot(vc.wo, hv);
            if (oh <= 0.0f) ok = false;
            else wi = hv * (2.0f * oh) - vc.wo;
        }
        if (ok && (dot(wi, vc.n) <= 0.0f || dot(wi, ngo) <= 0.0f)) ok = false;
        if (ok) { sh.pdf = bsdf_pdf(S, P, m, vc, wi); if (!(sh.pdf > 0.0f)) ok = false; }
    } else if (m.type == DPPT_MAT_SMOOTH_DIELECTRIC) {
        float eta = __ldg(P.ior + m.ior_index);
        float co = dot(vc.wo, vc.ng);
        vc.outside = co > 0.0f;
        float eo = vc.outside ? 1.0f : eta, et = vc.outside ? eta : 1.0f;
        float c = fabsf(co);
        float F = fresnel_unpolarized(c, eo, et);
        float r = eo / et, s2 = r * r * (1.0f - c * c);
        if (s2 >= 1.0f) F = 1.0f;
        if (U.u[0] < F) {
            sh.ev = 1u; vc.p_event = F;
            wi = vc.n * (2.0f * c) - vc.wo;
        } else {
            sh.ev = 2u; vc.p_event = 1.0f - F;
            float ct = sqrtf(1.0f - s2);
            wi = vc.n * (r * c - ct) - vc.wo * r;
        }
        sh.pdf = 1.0f;
    } else {
        wi = -vc.wo;
        sh.pdf = 1.0f;
    }
    sh.ok = ok;
    sh.wi = wi;
}

// Completes the vertex once the visibility of its light sample is known;
// returns true when the path continues.
template <int MT = -1, class Vis>
__device__ __forceinline__ bool walk_finish(const DScene& S, const DParams& P, Walk& w, VCtx& vc,
                                            const NeePending& ne, bool visible, const Shade& sh, Vis& vis) {
    unsigned neeflag = 2u;
    if (!sh.terminal) {
        vc.event = (int)sh.ev;
        vc.pdf = sh.pdf;
        if (ne.state != 2) {
            neeflag = 0u;
            if (ne.state == 1 && visible) {
                const DMat m = load_mat<MT>(S, vc.mat);
                float pl = ne.pl;
                float pb = bsdf_pdf(S, P, m, vc, ne.wl);
                float wm = pl * pl / (pl * pl + pb * pb);
                vc.nee = true; vc.nee_light = ne.l; vc.wl = ne.wl;
                vc.nee_w = ne.cx / pl * wm;
                neeflag = 1u;
            }
        }
    }
    w.sig = fnv(fnv(fnv(w.sig, (unsigned)vc.prim), sh.ev), neeflag);
    vc.scatter = !sh.terminal && sh.ok;
    vc.wi = sh.wi;
    ++w.nv;
    vis(vc);
    if (!vc.scatter) return false;
    float side = dot(sh.wi, vc.ng) >= 0.0f ? 1.0f : -1.0f;
    w.xprev = vc.x;
    w.o = vc.x + vc.ng * (side * S.eps);
    w.d = sh.wi;
    w.prev_delta = sh.delta;
    w.prev_pdf = sh.pdf;
    ++w.v;
    return true;
}

// Traces vertex w.v of the path and calls vis(vc) for it.  Returns true when
// the path continues with vertex w.v + 1.
template <class Vis, bool COUNT, bool NM = true, int MT = -1>
__device__ __forceinline__ bool walk_step(const DScene& S, const DParams& P, const DJob& J, unsigned long long pid,
                                          Walk& w, Vis& vis, unsigned* status, WorkCount* wc) {
    HitRec h;
    if (!trace_closest<COUNT>(S, w.o, w.d, h, status, wc)) return false;
    if (COUNT) wc->vertices++;
    VCtx vc;
    NeePending ne;
    Shade sh;
    walk_shade<NM, MT>(S, P, J, pid, w, h, vc, ne, sh);
    bool visible = false;
    if (ne.state == 1) visible = !trace_any<COUNT>(S, ne.o2, ne.dir, ne.tmax, status, wc);
    return walk_finish<MT>(S, P, w, vc, ne, visible, sh, vis);
}

// Gradient scatter of texel derivatives, chosen per launch (DScene::scatter_lane): either
// the lanes of a warp that add to the same element are grouped with __match_any_sync and
// one lane per group issues the atomic (the default: it keeps many warps that hit the same
// texels from serializing on them), or every lane issues its own atomic (faster when few
// lanes share texels, since the memory system already combines the lanes of one atomic
// instruction that hit the same address).
__device__ __forceinline__ void atomic_add_grouped(float* base, long long idx, float val) {
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, (unsigned long long)idx);
    const int lane = threadIdx.x & 31;
    float sum;
    if (peers == 0xffffffffu) {
        sum = val;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    } else {
        sum = 0.0f;
        for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, val, __ffs(m) - 1);
    }
    if (lane == __ffs(peers) - 1 && sum != 0.0f) atomicAdd(base + idx, sum);
}
// The block's scalar-gradient accumulators (sgrad_copies copies of each scalar), zeroed by
// all threads of the block at its start.
__device__ __forceinline__ void sgrad_zero(const DScene& S, float* sg) {
    const int n = sgrad_scalars(S) * sgrad_copies(S);
    for (int k = threadIdx.x; k < n; k += blockDim.x) sg[k] = 0.0f;
    __syncthreads();
}
__device__ __forceinline__ void sgrad_add(const DScene& S, float* sg, int k, float v) {
    const int copies = sgrad_copies(S);
    atomicAdd(sg + k * copies + (threadIdx.x & (copies - 1)), v);
}
// after the block's last addition: sums the copies (read in a rotated order, one bank per
// lane) and adds each nonzero scalar to its gradient with one global atomic
__device__ __forceinline__ void sgrad_flush(const DScene& S, const DGrads& G, const float* sg) {
    __syncthreads();
    const int nscal = sgrad_scalars(S), copies = sgrad_copies(S);
    const int nI = S.num_ior, nS = S.num_sheets, nT = sgrad_texel_base(S);
    for (int k = threadIdx.x; k < nscal; k += blockDim.x) {
        float v = 0.0f;
        for (int c = 0; c < copies; ++c) v += sg[k * copies + ((c + k) & (copies - 1))];
        if (v == 0.0f) continue;
        float* base;
        int off;
        if (k < nI) { base = G.ior; off = k; }
        else if (k < nI + nS) { base = G.sheet; off = k - nI; }
        else if (k < nT) { base = G.le; off = k - nI - nS; }
        else { base = G.tex; off = k - nT; }
        if (base) atomicAdd(base + off, v);
    }
}

// adds vals[c] * w[k] at tp.idx[k] + min(c, ch - 1) for the NC values and the four taps.
// UNROLL = false keeps the sixteen sites as a loop: the wavefront replay kernels are bound by
// instruction fetch, and sixteen inlined copies of the grouping code would enlarge them.
// The megakernels are bound by their thread-local cache and run faster unrolled.
// The same sums into the block's accumulators (DScene::tex_shared): no grouping, each lane adds
// to its own copy.
template <int NC>
__device__ __forceinline__ void scatter_taps_shared(const DScene& S, float* sg, const Taps& tp0, const float* vals,
                                                    int ch) {
    Taps tp = tp0;
#pragma unroll
    for (int k = 1; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < k; ++j)
            if (tp.w[k] != 0.0f && tp.idx[k] == tp.idx[j]) { tp.w[j] += tp.w[k]; tp.w[k] = 0.0f; }
    const int base = sgrad_texel_base(S);
#pragma unroll 1
    for (int c = 0; c < NC; ++c)
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            const float v = vals[c] * tp.w[k];
            if (v != 0.0f) sgrad_add(S, sg, base + (int)tp.idx[k] + min(c, ch - 1), v);
        }
}
template <int NC, bool UNROLL>
__device__ __forceinline__ void scatter_taps(float* g, const Taps& tp0, const float* vals, int ch, bool per_lane) {
    // taps on the same texel (a texture one or two texels wide, wrapped) are merged first,
    // and a zero value issues no atomic
    Taps tp = tp0;
#pragma unroll
    for (int k = 1; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < k; ++j)
            if (tp.w[k] != 0.0f && tp.idx[k] == tp.idx[j]) { tp.w[j] += tp.w[k]; tp.w[k] = 0.0f; }
    if (UNROLL) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float v = vals[c] * tp.w[k];
                const long long idx = tp.idx[k] + min(c, ch - 1);
                if (v == 0.0f) continue;
                if (per_lane) atomicAdd(g + idx, v);
                else atomic_add_grouped(g, idx, v);
            }
    } else {
#pragma unroll 1
        for (int c = 0; c < NC; ++c)
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                const float v = vals[c] * tp.w[k];
                const long long idx = tp.idx[k] + min(c, ch - 1);
                if (v == 0.0f) continue;
                if (per_lane) atomicAdd(g + idx, v);
                else atomic_add_grouped(g, idx, v);
            }
    }
}

// ================================================================== per-vertex actions
// Where a path's cached E_v / compact W_v live: thread-local arrays (megakernel) or one
// record per (vertex, path) in global memory (wavefront).  Both hold W_v as 19 floats in
// the order ri.c, ri.s, ro.c, ro.s, A[3], B[3], C[3], S[3], D[3].
__device__ __forceinline__ void pack_w(const Compact<float>& W, float o[20]) {
    o[0] = W.ri.c; o[1] = W.ri.s; o[2] = W.ro.c; o[3] = W.ro.s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o[4 + c] = W.A[c]; o[7 + c] = W.B[c]; o[10 + c] = W.C[c]; o[13 + c] = W.S[c]; o[16 + c] = W.D[c];
    }
    o[19] = 0.0f;
}
__device__ __forceinline__ void unpack_w(const float o[19], Compact<float>& W) {
    W.ri = {o[0], o[1]}; W.ro = {o[2], o[3]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        W.A[c] = o[4 + c]; W.B[c] = o[7 + c]; W.C[c] = o[10 + c]; W.S[c] = o[13 + c]; W.D[c] = o[16 + c];
    }
}

// The megakernels' thread-local cache: per vertex E_v in three float4s and W_v in five (19
// floats and a pad), so that a vertex moves with eight vector accesses.
template <int MAXD>
struct LocalCache {
    float4 (*cE)[3];
    float4 (*cW)[5];
    static constexpr int cap = MAXD;
    static constexpr bool kUnrollScatter = true;
    __device__ __forceinline__ void put(int v, const float E[12], const Compact<float>& W) const {
        float o[20];
        pack_w(W, o);
#pragma unroll
        for (int k = 0; k < 3; ++k) cE[v][k] = make_float4(E[4 * k], E[4 * k + 1], E[4 * k + 2], E[4 * k + 3]);
#pragma unroll
        for (int k = 0; k < 5; ++k) cW[v][k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
    }
    __device__ __forceinline__ void get_w(int v, Compact<float>& W) const {
        float o[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 t = cW[v][k];
            o[4 * k] = t.x; o[4 * k + 1] = t.y; o[4 * k + 2] = t.z; o[4 * k + 3] = t.w;
        }
        unpack_w(o, W);
    }
    __device__ __forceinline__ void get_e(int v, float e[12]) const {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = cE[v][k];
            e[4 * k] = t.x; e[4 * k + 1] = t.y; e[4 * k + 2] = t.z; e[4 * k + 3] = t.w;
        }
    }
    __device__ __forceinline__ void put_e(int v, const float e[12]) const {
#pragma unroll
        for (int k = 0; k < 3; ++k) cE[v][k] = make_float4(e[4 * k], e[4 * k + 1], e[4 * k + 2], e[4 * k + 3]);
    }
};

// A vertex of the wavefront's global cache: one 144-byte record per (vertex, path), so a
// path's record stays whole however sparse the live paths of an iteration become (nine
// float4s: E_v 12 floats, compact W_v 19, one word with the visibility of the vertex's
// light sample and the vertex's replay bin, the closest hit of the ray that made the
// vertex: t, b1, b2, code).  The replay reads the hit and the visibility instead of
// tracing the ray and the shadow ray again (it would find exactly the same hits).
constexpr int kWfCacheComps = 36;
constexpr int kWfVisComp = 31;
constexpr int kWfHitComp = 32;
// The sweep schedule's records keep only what the replay reads: 64 bytes per (vertex, path),
// the suffix L_v (0-11) and the hit (12-15), so that its writes fill whole 32-byte sectors;
// the visibility words are in a plane of their own.
constexpr int kSweepRecFloats = 16;
constexpr int kSweepHitComp = 12;
struct GlobalCache {
    float* base;
    long long Q, q;
    int cap;
    int stride;     // floats per record: kWfCacheComps, or kSweepRecFloats (suffix first in both)
    static constexpr bool kUnrollScatter = false;
    __device__ __forceinline__ float4* rec(int v) const {
        return reinterpret_cast<float4*>(base + ((long long)v * Q + q) * stride);
    }
    // writes E_v and W_v (and a zero visibility, which the caller sets afterwards)
    __device__ __forceinline__ void put(int v, const float E[12], const Compact<float>& W) const {
        float o[20];
        pack_w(W, o);
        float4* r = rec(v);
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = make_float4(E[4 * k], E[4 * k + 1], E[4 * k + 2], E[4 * k + 3]);
#pragma unroll
        for (int k = 0; k < 5; ++k) r[3 + k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
    }
    __device__ __forceinline__ void get_w(int v, Compact<float>& W) const {
        const float4* r = rec(v);
        float o[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 t = r[3 + k];
            o[4 * k] = t.x; o[4 * k + 1] = t.y; o[4 * k + 2] = t.z; o[4 * k + 3] = t.w;
        }
        unpack_w(o, W);
    }
    __device__ __forceinline__ void get_e(int v, float e[12]) const {
        const float4* r = rec(v);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = r[k];
            e[4 * k] = t.x; e[4 * k + 1] = t.y; e[4 * k + 2] = t.z; e[4 * k + 3] = t.w;
        }
    }
    __device__ __forceinline__ void put_e(int v, const float e[12]) const {
        float4* r = rec(v);
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = make_float4(e[4 * k], e[4 * k + 1], e[4 * k + 2], e[4 * k + 3]);
    }
};

// The backward fold of cached vertices top .. 0 (Sec. 4.3: L_v = E_v + W_v L_{v+1}): L enters
// as the suffix of vertex top + 1 and leaves as that of vertex 0; the adjoint keeps each
// suffix of a vertex v >= 1 in the cache for the replay, which reads L_{v+1}.
template <class Cache>
__device__ __forceinline__ void fold_cached(const Cache& C, int top, bool adjoint, float L[12]) {
    for (int v = top; v >= 0; --v) {
        Compact<float> W;
        C.get_w(v, W);
        float e[12];
        C.get_e(v, e);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float y[4];
            compact_apply(W, c, &L[4 * c], y);
#pragma unroll
            for (int k = 0; k < 4; ++k) L[4 * c + k] = e[4 * c + k] + y[k];
        }
        if (adjoint && v >= 1) C.put_e(v, L);
    }
}

// Local vector-Jacobian products of one dual-number evaluation of a replayed vertex:
// per channel J_c = a_c^T (W_c L_c + f_c Le_c nee_w) (W and the NEE operator f from
// eval_vertex<D3>, Ln the suffix L[v+1]); returns the three slots' derivatives, the third
// per channel.
template <class DT>
__device__ __forceinline__ void local_vjp(const DScene& S, const DParams& P, const VCtx& vc, const Compact<DT>& W,
                                          const Compact<DT>& f, const Rot<float>& Rle, const float Ln[3][4],
                                          const float a[3][4], float& g0, float& g1, float g2[3]) {
    g0 = g1 = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        DT x[4] = {DT(Ln[c][0]), DT(Ln[c][1]), DT(Ln[c][2]), DT(Ln[c][3])};
        DT y[4];
        compact_apply(W, c, x, y);
        DT J = y[0] * a[c][0] + y[1] * a[c][1] + y[2] * a[c][2] + y[3] * a[c][3];
        if (vc.nee) {
            const float* le = P.le + 12 * vc.nee_light + 4 * c;
            float lv[4] = {__ldg(le), __ldg(le + 1), __ldg(le + 2), __ldg(le + 3)};
            rot_apply(Rle, lv);
            DT xe[4] = {DT(lv[0] * vc.nee_w), DT(lv[1] * vc.nee_w), DT(lv[2] * vc.nee_w), DT(lv[3] * vc.nee_w)};
            DT ye[4];
            compact_apply(f, c, xe, ye);
            J = J + ye[0] * a[c][0] + ye[1] * a[c][1] + ye[2] * a[c][2] + ye[3] * a[c][3];
        }
        g0 += dslot0(J);
        g1 += dslot1(J);
        g2[c] = dslot2(J);
    }
}

// The normal map's texel derivatives at a normal-mapped replayed vertex: a second dual
// evaluation whose slots carry the three components of n = 2 c - 1.  Not inlined: it runs
// at normal-mapped vertices only and would otherwise raise the register pressure of every
// replay kernel that may meet one.
template <int MT>
__device__ __noinline__ void normal_map_vjp(const DScene& S, const DParams& P, const DGrads& G, const VCtx& vc,
                                            const Rot<float> Rle, const float Ln[3][4], const float a[3][4]) {
    const DMat m = load_mat<MT>(S, vc.mat);
    f3 nN, nT, nB;
    if (!nmap_frame(S, m, vc, nN, nT, nB)) return;
    float En[3][4];
    Compact<D3> Wn, fn;
    eval_vertex<D3, MT, true, true>(S, P, vc, En, Wn, &fn);
    float h0, h1, h2[3];
    local_vjp(S, P, vc, Wn, fn, Rle, Ln, a, h0, h1, h2);
    const Taps tp = tex_taps(S.tex[m.normal_tex], vc.tu, vc.tv);
    const float gn[3] = {2.0f * h0, 2.0f * h1, 2.0f * (h2[0] + h2[1] + h2[2])};
    scatter_taps<3, false>(G.tex, tp, gn, 3, S.scatter_lane != 0);
}

// The replayed vertex's local vector-Jacobian product, scattered into the gradients, then
// the adjoint row's advance a^T <- a^T W_v.  W and f come from eval_vertex<D3> with the
// material's own slots.  At a normal-mapped vertex a second evaluation, whose slots carry
// the map value n, gives the normal map's texel derivatives.
template <int MT = -1, bool NM = true, bool UNROLL = true, class DT = D3>
__device__ __forceinline__ void replay_vjp(const DScene& S_, const DParams& P_, const DGrads& G_, float* sgrad,
                                           const VCtx& vc, const Compact<DT>& W, const Compact<DT>& f,
                                           const float Ln[3][4], float a[3][4]) {
    const DScene* S = &S_;
    const DGrads* G = &G_;
    const DMat m = load_mat<MT>(S_, vc.mat);
    Rot<float> Rle = {1.0f, 0.0f};
    if (vc.nee) Rle = emitter_rot(load_light(*S, vc.nee_light), -vc.wl);
    float g_slot0, g_eta, g_alb[3];
    local_vjp(S_, P_, vc, W, f, Rle, Ln, a, g_slot0, g_eta, g_alb);
    // emitter Stokes gradients (linear): w R^T a for a hit, nee_w R^T f^T a for NEE
    if (vc.emit || vc.nee) {
        const int base = S->num_ior + S->num_sheets;
        Rot<float> Re = {1.0f, 0.0f};
        if (vc.emit) Re = emitter_rot(load_light(*S, vc.light), vc.wo);
        Compact<float> fv;
        if (vc.nee) fv = compact_value(f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (vc.emit) {
                float g[4] = {a[c][0], a[c][1], a[c][2], a[c][3]};
                rot_apply_row(Re, g);
                for (int k = 0; k < 4; ++k)
                    if (g[k] != 0.0f) sgrad_add(*S, sgrad, base + 12 * vc.light + 4 * c + k, g[k] * vc.w_emit);
            }
            if (vc.nee) {
                float g[4] = {a[c][0], a[c][1], a[c][2], a[c][3]};
                compact_row(fv, c, g);
                rot_apply_row(Rle, g);
                for (int k = 0; k < 4; ++k)
                    if (g[k] != 0.0f) sgrad_add(*S, sgrad, base + 12 * vc.nee_light + 4 * c + k, g[k] * vc.nee_w);
            }
        }
    }
    // parameter scatter
    if (m.type == DPPT_MAT_SMOOTH_DIELECTRIC || m.type == DPPT_MAT_PLASTIC_GGX) {
        if (g_eta != 0.0f) sgrad_add(*S, sgrad, m.ior_index, g_eta);
    }
    if (m.type == DPPT_MAT_POLARIZER_SHEET || m.type == DPPT_MAT_RETARDER_SHEET) {
        if (g_slot0 != 0.0f) sgrad_add(*S, sgrad, S->num_ior + m.sheet_index, g_slot0);
    }
    if (G->tex) {
        if ((m.type == DPPT_MAT_CONDUCTOR_GGX || m.type == DPPT_MAT_PLASTIC_GGX) && S->tex[m.rough_tex].pad) {
            Taps tp = tex_taps(S->tex[m.rough_tex], vc.tu, vc.tv);
            if (S->tex_shared) scatter_taps_shared<1>(*S, sgrad, tp, &g_slot0, 1);
            else scatter_taps<1, UNROLL>(G->tex, tp, &g_slot0, 1, S->scatter_lane != 0);
        }
        if (m.albedo_tex >= 0 && (m.type == DPPT_MAT_DIFFUSE || m.type == DPPT_MAT_CONDUCTOR_GGX ||
                                  m.type == DPPT_MAT_PLASTIC_GGX) && S->tex[m.albedo_tex].pad) {
            DTex t = S->tex[m.albedo_tex];
            Taps tp = tex_taps(t, vc.tu, vc.tv);
            if (S->tex_shared) scatter_taps_shared<3>(*S, sgrad, tp, g_alb, t.ch);
            else scatter_taps<3, UNROLL>(G->tex, tp, g_alb, t.ch, S->scatter_lane != 0);
        }
    }
    if constexpr (NM) {
        if (G->tex && m.normal_tex >= 0 && S->tex[m.normal_tex].pad) normal_map_vjp<MT>(S_, P_, G_, vc, Rle, Ln, a);
    }
    // advance the adjoint row through the value of W_i
    Compact<float> Wv = compact_value(W);
#pragma unroll
    for (int c = 0; c < 3; ++c) compact_row(Wv, c, a[c]);
}

// Pass 0 caches E_v and the compact W_v of every vertex after which the path goes on
// (the last vertex has L[n] = E_n, so its W is never needed and its E stays in
// registers); the backward fold overwrites E_v with the suffix L[v] where the replay
// will read it (the adjoint's vertices 1..n-1).  Pass 1 (adjoint only) replays the
// vertex with dual numbers.
template <class Cache, int MT = -1, bool NM = true>
struct PathVis {
    const DScene* S;
    const DParams* P;
    const DGrads* G;
    float* sgrad;       // shared scalar-gradient accumulators [ior | sheet | le]
    Cache C;
    float a[3][4];      // adjoint row a^T = dI^T C R_cam W_1 ... W_{v-1}
    float lastE[12];    // emission at the path's last vertex
    int n, i, phase;
    bool has_last, adjoint;

    __device__ __forceinline__ void operator()(const VCtx& vc) {
        if (phase == 0) {
            if (n >= C.cap) return;
            float E[3][4];
            Compact<float> W;
            eval_vertex<float, MT, NM>(*S, *P, vc, E, W, nullptr);
            if (!vc.scatter) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) lastE[4 * c + k] = E[c][k];
                has_last = true;
                ++n;
                return;
            }
            C.put(n, &E[0][0], W);
            ++n;
            return;
        }
        if (i >= n) return;
        replay_vertex(vc);
        ++i;
    }

    // backward fold of the cached vertices into suffixes; returns L[1] in L0
    __device__ __forceinline__ void fold(float L0[12]) {
#pragma unroll
        for (int k = 0; k < 12; ++k) L0[k] = has_last ? lastE[k] : 0.0f;
        int v = n - 1;
        if (has_last) {
            if (adjoint && v >= 1) C.put_e(v, L0);
            --v;
        }
        fold_cached(C, v, adjoint, L0);
    }

    __device__ void replay_vertex(const VCtx& vc) {
        // a diffuse vertex has one differentiable material value (its albedo), a rough
        // conductor two (roughness and albedo tint): duals with only those slots
        using DT = typename std::conditional<MT == DPPT_MAT_DIFFUSE, D1,
                   typename std::conditional<MT == DPPT_MAT_CONDUCTOR_GGX, D2, D3>::type>::type;
        float E[3][4];
        Compact<DT> W, f;
        eval_vertex<DT, MT, NM>(*S, *P, vc, E, W, &f);
        float Ln[3][4];
        if (i + 1 < n) {
            C.get_e(i + 1, &Ln[0][0]);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) Ln[k >> 2][k & 3] = 0.0f;
        }
        replay_vjp<MT, NM, Cache::kUnrollScatter, DT>(*S, *P, *G, sgrad, vc, W, f, Ln, a);
    }
};

__device__ __forceinline__ int find_job(const JobTable& T, long long chunk) {
    int j = 0;
    while (j + 1 < T.njobs && T.job[j + 1].chunk_begin <= chunk) ++j;
    return j;
}

// Adds one path's raw Stokes (already divided by spp) to its pixel.  Called by
// all 32 lanes of the warp (inactive lanes pass zeros); the job is uniform
// across the block.  red_mode 0: spp a power of two <= 32, a segment of lanes
// holds whole pixels -> shuffle sum and one plain store; 1: spp a power-of-two
// multiple of 32 -> warp sum and one atomic per warp; 2: one atomic per path.
__device__ __forceinline__ void pixel_reduce(const DJob& J, float* dst, long long p, bool active, float v[12]) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (J.red_mode == 0) {
        for (int off = 1; off < J.spp; off <<= 1)
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] += __shfl_xor_sync(FULL, v[k], off);
        if (active && (lane % J.spp) == 0) {
            float4* o = reinterpret_cast<float4*>(dst + (p / J.spp) * 12);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
            o[2] = make_float4(v[8], v[9], v[10], v[11]);
        }
    } else if (J.red_mode == 1) {
        for (int off = 1; off < 32; off <<= 1)
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] += __shfl_xor_sync(FULL, v[k], off);
        if (active && lane == 0)
            for (int k = 0; k < 12; ++k) atomicAdd(dst + (p / J.spp) * 12 + k, v[k]);
    } else if (active) {
        for (int k = 0; k < 12; ++k) atomicAdd(dst + (p / J.spp) * 12 + k, v[k]);
    }
}

// ================================================================== megakernel
// NM = false compiles the normal-map code out: the adjoint is launched with it only for
// scenes that have normal maps (their second dual evaluation would otherwise raise the
// register pressure of every adjoint).
template <int MAXD, int MODE, bool COUNT, bool NM = true, int MT = -1>
__global__ void __launch_bounds__(256, MODE == 1 ? DPPT_MIN_BLOCKS_ADJOINT : DPPT_MIN_BLOCKS_PRIMAL)
k_trace(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T,
        unsigned long long* counter, unsigned* status, int persistent, unsigned long long* work) {
    extern __shared__ float sgrad[];
    __shared__ long long s_chunk;
    if (MODE == 1) sgrad_zero(S, sgrad);
    float4 cE[MAXD][3];
    float4 cW[MAXD][5];
    WorkCount wc = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    unsigned long long paths_done = 0;
    long long chunk = blockIdx.x;
    for (;;) {
        if (persistent) {
            __syncthreads();
            if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(counter, 1ULL);
            __syncthreads();
            chunk = s_chunk;
        }
        if (chunk >= T.total_chunks) break;
        const DJob& J = T.job[find_job(T, chunk)];
        const long long p = (chunk - J.chunk_begin) * blockDim.x + threadIdx.x;
        const bool active = p < J.npaths;
        float raw[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) raw[k] = 0.0f;
        if (active) {
            const long long pix = p / J.spp;
            PathVis<LocalCache<MAXD>, MT, NM> vis;
            vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad;
            vis.C.cE = cE; vis.C.cW = cW;
            vis.n = 0; vis.i = 0; vis.has_last = false; vis.adjoint = MODE == 1;
            Walk w;
            const int passes = MODE == 1 ? 2 : 1;
            // pass 0 caches E_i and W_i; pass 1 replays the same path through the same call site
#pragma unroll 1
            for (int phase = 0; phase < passes; ++phase) {
                vis.phase = phase;
                walk_begin(S, J, (unsigned long long)p, pix, w);
                while (walk_step<PathVis<LocalCache<MAXD>, MT, NM>, COUNT, NM, MT>(S, P, J, (unsigned long long)p, w, vis,
                                                                               status, &wc)) {
                }
                if (phase == 0) {
                    float L0[12];
                    vis.fold(L0);
                    Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
                    const float inv = 1.0f / (float)J.spp;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
                        rot_apply(Rc, v);
#pragma unroll
                        for (int k = 0; k < 4; ++k) raw[4 * c + k] = v[k] * inv;
                    }
                    if (MODE == 1) {
                        if (vis.n == 0) break;
                        const float* ds = J.dS + pix * 12;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float av[4] = {__ldg(ds + 4 * c) * inv, __ldg(ds + 4 * c + 1) * inv,
                                           __ldg(ds + 4 * c + 2) * inv, __ldg(ds + 4 * c + 3) * inv};
                            rot_apply_row(Rc, av);
#pragma unroll
                            for (int k = 0; k < 4; ++k) vis.a[c][k] = av[k];
                        }
                    }
                }
            }
            if (J.sig) J.sig[p] = fnv(w.sig, (unsigned)w.nv);
            ++paths_done;
        }
        if (J.raw) {
            __syncwarp();
            pixel_reduce(J, J.raw, p, active, raw);
        }
        if (!persistent) break;
    }
    if (COUNT) {
        atomicAdd(work + 0, paths_done);
        atomicAdd(work + 1, (unsigned long long)wc.vertices);
        atomicAdd(work + 2, (unsigned long long)wc.rays);
        atomicAdd(work + 3, (unsigned long long)wc.shadow_rays);
        atomicAdd(work + 4, (unsigned long long)wc.nodes);
        atomicAdd(work + 5, (unsigned long long)wc.shadow_nodes);
        atomicAdd(work + 6, (unsigned long long)wc.tri_tests);
        atomicAdd(work + 7, (unsigned long long)wc.shadow_tri_tests);
        atomicAdd(work + 8, (unsigned long long)wc.sph_tests);
        atomicAdd(work + 9, (unsigned long long)wc.shadow_sph_tests);
    }
    if (MODE == 1) sgrad_flush(S, G, sgrad);
}

// one translation unit per cache depth instantiates its kernels and launchers
#define DPPT_TRACE_BUCKET(B)                                                                                        \
    cudaError_t launch_trace_##B(int mode, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,  \
                                 const LaunchCfg& L, unsigned long long* counter, unsigned* status,              \
                                 unsigned long long* work, cudaStream_t st) {                                    \
        const int pers = L.schedule == DPPT_SCHED_PERSISTENT;                                                    \
        long long g = pers ? L.grid : T.total_chunks;                                                            \
        if (g <= 0) return cudaSuccess;                                                                          \
        if (g > 0x7fffffffLL) g = 0x7fffffffLL;                                                                  \
        if (mode == 0) {                                                                                         \
            if (S.tri_tan)                                                                                       \
                k_trace<B, 0, false, true><<<(int)g, L.block, 0, st>>>(S, P, G, T, counter, status, pers, nullptr); \
            else if ((S.mat_types & ~kDiffuseDielectricTypes) == 0)                                              \
                k_trace<B, 0, false, false, type_mask_mt(kDiffuseDielectricTypes)>                              \
                    <<<(int)g, L.block, 0, st>>>(S, P, G, T, counter, status, pers, nullptr);                    \
            else                                                                                                 \
                k_trace<B, 0, false, false><<<(int)g, L.block, 0, st>>>(S, P, G, T, counter, status, pers, nullptr);\
        } else if (mode == 1) {                                                                                  \
            size_t sm = sgrad_bytes(S);                                                                         \
            if (S.tri_tan)                                                                                       \
                k_trace<B, 1, false, true><<<(int)g, L.block, sm, st>>>(S, P, G, T, counter, status, pers, nullptr); \
            else                                                                                                 \
                k_trace<B, 1, false, false><<<(int)g, L.block, sm, st>>>(S, P, G, T, counter, status, pers, nullptr);\
        } else                                                                                                   \
            k_trace<B, 0, true><<<(int)g, L.block, 0, st>>>(S, P, G, T, counter, status, pers, work);             \
        return cudaGetLastError();                                                                               \
    }                                                                                                            \
    /* the attributes are those of the kernels without normal-map code (the same launch     */                  \
    /* bounds as the ones with it)                                                          */                  \
    cudaError_t trace_attributes_##B(int mode, cudaFuncAttributes* a) {                                         \
        return cudaFuncGetAttributes(a, mode == 0 ? reinterpret_cast<const void*>(&k_trace<B, 0, false, false>)   \
                                                  : reinterpret_cast<const void*>(&k_trace<B, 1, false, false>)); \
    }                                                                                                            \
    int trace_occupancy_##B(int mode, int block, size_t smem) {                                                  \
        int nb = 0;                                                                                              \
        const void* f = mode == 0 ? reinterpret_cast<const void*>(&k_trace<B, 0, false, false>)                   \
                                  : reinterpret_cast<const void*>(&k_trace<B, 1, false, false>);                 \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem) != cudaSuccess) return 0;          \
        return nb;                                                                                               \
    }

}  // namespace dppt
