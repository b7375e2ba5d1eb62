// Device math for the polarized path tracer: vectors, dual numbers, the
// counter-based generator, Stokes frames and rotators, Fresnel Mueller blocks
// and the GGX microfacet terms.  Everything is FP32 in registers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dppt {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;

// ------------------------------------------------------------------ vectors
struct f3 { float x, y, z; };
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator-(f3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float len(f3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ f3 normalize(f3 a) { return a * (1.0f / len(a)); }
__device__ __forceinline__ f3 ld3(const float* p) { return {p[0], p[1], p[2]}; }

// First tangent of the branchless orthonormal basis of Duff et al. (2017);
// (t1, n x t1, n) is right handed.  It is the x axis of the Stokes frame of
// light propagating along n, and the sampling frame of a surface normal.
__device__ __forceinline__ f3 onb_t1(f3 n) {
    float sg = copysignf(1.0f, n.z);
    float a = -1.0f / (sg + n.z);
    float b = n.x * n.y * a;
    return {1.0f + sg * n.x * n.x * a, sg * b, -sg * n.x};
}
__device__ __forceinline__ f3 onb_t2(f3 n) {
    float sg = copysignf(1.0f, n.z);
    float a = -1.0f / (sg + n.z);
    float b = n.x * n.y * a;
    return {b, sg + n.y * n.y * a, -n.y};
}

// ------------------------------------------------------------------ dual numbers
// Value plus three directional derivatives.  In the adjoint replay slot 0 is
// the GGX roughness (or a sheet's axis angle), slot 1 the index of refraction,
// slot 2 the albedo/tint of the channel being evaluated.
struct D3 {
    float v, d0, d1, d2;
    __device__ __forceinline__ D3() {}
    __device__ __forceinline__ D3(float x) : v(x), d0(0.f), d1(0.f), d2(0.f) {}
    __device__ __forceinline__ D3(float x, float a, float b, float c) : v(x), d0(a), d1(b), d2(c) {}
};
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
__device__ __forceinline__ D3 operator-(D3 a) { return {-a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ D3 operator*(D3 a, D3 b) {
    return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
__device__ __forceinline__ D3 operator*(D3 a, float s) { return {a.v * s, a.d0 * s, a.d1 * s, a.d2 * s}; }
__device__ __forceinline__ D3 operator*(float s, D3 a) { return a * s; }
__device__ __forceinline__ D3 operator+(D3 a, float s) { return {a.v + s, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ D3 operator+(float s, D3 a) { return a + s; }
__device__ __forceinline__ D3 operator-(D3 a, float s) { return {a.v - s, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ D3 operator-(float s, D3 a) { return {s - a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ D3 operator/(D3 a, D3 b) {
    float r = 1.0f / b.v, q = a.v * r;
    return {q, (a.d0 - q * b.d0) * r, (a.d1 - q * b.d1) * r, (a.d2 - q * b.d2) * r};
}
__device__ __forceinline__ D3 operator/(D3 a, float s) { return a * (1.0f / s); }
__device__ __forceinline__ D3 operator/(float s, D3 b) {
    float r = 1.0f / b.v, q = s * r;
    return {q, -q * b.d0 * r, -q * b.d1 * r, -q * b.d2 * r};
}
__device__ __forceinline__ D3 tsqrt(D3 a) {
    float s = sqrtf(a.v), h = 0.5f / s;
    return {s, a.d0 * h, a.d1 * h, a.d2 * h};
}
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(D3 a) { return a.v; }
__device__ __forceinline__ D3 tcos(D3 a) { float s, c; sincosf(a.v, &s, &c); return {c, -s * a.d0, -s * a.d1, -s * a.d2}; }
__device__ __forceinline__ D3 tsin(D3 a) { float s, c; sincosf(a.v, &s, &c); return {s, c * a.d0, c * a.d1, c * a.d2}; }
// One-slot dual number: a value and its derivative with respect to one parameter (the
// replay of a diffuse vertex, whose only differentiable material value is its albedo).
struct D1 {
    float v, d;
    __device__ __forceinline__ D1() {}
    __device__ __forceinline__ D1(float x) : v(x), d(0.f) {}
    __device__ __forceinline__ D1(float x, float a) : v(x), d(a) {}
};
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator-(D1 a) { return {-a.v, -a.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator*(D1 a, float s) { return {a.v * s, a.d * s}; }
__device__ __forceinline__ D1 operator*(float s, D1 a) { return a * s; }
__device__ __forceinline__ D1 operator+(D1 a, float s) { return {a.v + s, a.d}; }
__device__ __forceinline__ D1 operator+(float s, D1 a) { return a + s; }
__device__ __forceinline__ D1 operator-(D1 a, float s) { return {a.v - s, a.d}; }
__device__ __forceinline__ D1 operator-(float s, D1 a) { return {s - a.v, -a.d}; }
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
    float r = 1.0f / b.v, q = a.v * r;
    return {q, (a.d - q * b.d) * r};
}
__device__ __forceinline__ D1 operator/(D1 a, float s) { return a * (1.0f / s); }
__device__ __forceinline__ D1 operator/(float s, D1 b) {
    float r = 1.0f / b.v, q = s * r;
    return {q, -q * b.d * r};
}
__device__ __forceinline__ D1 tsqrt(D1 a) {
    float s = sqrtf(a.v);
    return {s, a.d * (0.5f / s)};
}
__device__ __forceinline__ float val(D1 a) { return a.v; }
__device__ __forceinline__ D1 tcos(D1 a) { float s, c; sincosf(a.v, &s, &c); return {c, -s * a.d}; }
__device__ __forceinline__ D1 tsin(D1 a) { float s, c; sincosf(a.v, &s, &c); return {s, c * a.d}; }
// Two-slot dual number: derivatives with respect to slots 0 and 2 (the replay of a rough
// conductor: roughness and albedo tint; its complex index of refraction is a constant).
struct D2 {
    float v, d0, d2;
    __device__ __forceinline__ D2() {}
    __device__ __forceinline__ D2(float x) : v(x), d0(0.f), d2(0.f) {}
    __device__ __forceinline__ D2(float x, float a, float c) : v(x), d0(a), d2(c) {}
};
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return {a.v + b.v, a.d0 + b.d0, a.d2 + b.d2}; }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) { return {a.v - b.v, a.d0 - b.d0, a.d2 - b.d2}; }
__device__ __forceinline__ D2 operator-(D2 a) { return {-a.v, -a.d0, -a.d2}; }
__device__ __forceinline__ D2 operator*(D2 a, D2 b) { return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d2 * b.v + a.v * b.d2}; }
__device__ __forceinline__ D2 operator*(D2 a, float s) { return {a.v * s, a.d0 * s, a.d2 * s}; }
__device__ __forceinline__ D2 operator*(float s, D2 a) { return a * s; }
__device__ __forceinline__ D2 operator+(D2 a, float s) { return {a.v + s, a.d0, a.d2}; }
__device__ __forceinline__ D2 operator+(float s, D2 a) { return a + s; }
__device__ __forceinline__ D2 operator-(D2 a, float s) { return {a.v - s, a.d0, a.d2}; }
__device__ __forceinline__ D2 operator-(float s, D2 a) { return {s - a.v, -a.d0, -a.d2}; }
__device__ __forceinline__ D2 operator/(D2 a, D2 b) {
    float r = 1.0f / b.v, q = a.v * r;
    return {q, (a.d0 - q * b.d0) * r, (a.d2 - q * b.d2) * r};
}
__device__ __forceinline__ D2 operator/(D2 a, float s) { return a * (1.0f / s); }
__device__ __forceinline__ D2 operator/(float s, D2 b) {
    float r = 1.0f / b.v, q = s * r;
    return {q, -q * b.d0 * r, -q * b.d2 * r};
}
__device__ __forceinline__ D2 tsqrt(D2 a) {
    float s = sqrtf(a.v), h = 0.5f / s;
    return {s, a.d0 * h, a.d2 * h};
}
__device__ __forceinline__ float val(D2 a) { return a.v; }
__device__ __forceinline__ D2 tcos(D2 a) { float s, c; sincosf(a.v, &s, &c); return {c, -s * a.d0, -s * a.d2}; }
__device__ __forceinline__ D2 tsin(D2 a) { float s, c; sincosf(a.v, &s, &c); return {s, c * a.d0, c * a.d2}; }
__device__ __forceinline__ float tcos(float a) { return cosf(a); }
__device__ __forceinline__ float tsin(float a) { return sinf(a); }

// ------------------------------------------------------------------ Philox4x64-10
// Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = 0xD2E7470EE14C6C93ULL * c[0];
        const uint64_t hi0 = __umul64hi(0xD2E7470EE14C6C93ULL, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ULL * c[2];
        const uint64_t hi1 = __umul64hi(0xCA5A826395121157ULL, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ULL; k1 += 0xBB67AE8584CAA73BULL;
    }
}
// Eight uniforms in [0, 1) with 24 random bits each (exact in float).
struct U8 { float u[8]; };
__device__ __forceinline__ U8 draw8(uint64_t k0, uint64_t k1, uint64_t path, uint32_t vertex) {
    uint64_t c[4] = {path, (uint64_t)vertex, 0ULL, 0ULL};
    philox4x64_10(c, k0, k1);
    U8 r;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        r.u[2 * i] = (float)((uint32_t)c[i] >> 8) * 5.9604644775390625e-08f;
        r.u[2 * i + 1] = (float)((uint32_t)(c[i] >> 32) >> 8) * 5.9604644775390625e-08f;
    }
    return r;
}

// ------------------------------------------------------------------ Stokes rotators
// Rot{c, s} re-expresses a Stokes vector from a frame with x axis x_from to one
// with x axis x_to (both normal to the propagation direction p, y = p x x):
// s1' = c s1 + s s2, s2' = -s s1 + c s2 with c = cos 2phi, s = sin 2phi and
// x_to = cos(phi) x_from + sin(phi) y_from.
template <class T> struct Rot { T c, s; };
__device__ __forceinline__ Rot<float> rot_between(f3 p, f3 x_from, f3 x_to) {
    f3 y_from = cross(p, x_from);
    float cf = dot(x_from, x_to), sf = dot(y_from, x_to);
    float inv = 1.0f / (cf * cf + sf * sf);
    return {(cf * cf - sf * sf) * inv, 2.0f * cf * sf * inv};
}
template <class T> __device__ __forceinline__ Rot<T> rot_to_param(f3 p, f3 x_from, const T xt[3]) {
    f3 y_from = cross(p, x_from);
    T cf = xt[0] * x_from.x + xt[1] * x_from.y + xt[2] * x_from.z;
    T sf = xt[0] * y_from.x + xt[1] * y_from.y + xt[2] * y_from.z;
    T n2 = cf * cf + sf * sf;
    return {(cf * cf - sf * sf) / n2, (cf * sf * 2.0f) / n2};
}
template <class T> __device__ __forceinline__ Rot<T> rot_from_param(f3 p, const T xf[3], f3 x_to) {
    T yf[3] = {xf[2] * p.y - xf[1] * p.z, xf[0] * p.z - xf[2] * p.x, xf[1] * p.x - xf[0] * p.y};
    T cf = xf[0] * x_to.x + xf[1] * x_to.y + xf[2] * x_to.z;
    T sf = yf[0] * x_to.x + yf[1] * x_to.y + yf[2] * x_to.z;
    T n2 = cf * cf + sf * sf;
    return {(cf * cf - sf * sf) / n2, (cf * sf * 2.0f) / n2};
}
// column vector:  v <- R v
template <class T, class V> __device__ __forceinline__ void rot_apply(const Rot<T>& r, V v[4]) {
    V a = r.c * v[1] + r.s * v[2];
    V b = r.c * v[2] - r.s * v[1];
    v[1] = a; v[2] = b;
}
// row vector:  a^T <- a^T R
template <class T, class V> __device__ __forceinline__ void rot_apply_row(const Rot<T>& r, V v[4]) {
    V a = r.c * v[1] - r.s * v[2];
    V b = r.s * v[1] + r.c * v[2];
    v[1] = a; v[2] = b;
}

// ------------------------------------------------------------------ complex
template <class T> struct Cx { T re, im; };
template <class T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> __device__ __forceinline__ Cx<T> cdiv(Cx<T> a, Cx<T> b) {
    T d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// principal root, written without cancellation; -x + 0i -> +i sqrt(x)
template <class T> __device__ __forceinline__ Cx<T> csqrt(Cx<T> z) {
    T r = tsqrt(z.re * z.re + z.im * z.im);
    if (val(r) == 0.0f) return {T(0.0f), T(0.0f)};
    if (val(z.re) >= 0.0f) {
        T t = tsqrt((r + z.re) * 0.5f);
        return {t, z.im / (t * 2.0f)};
    }
    T t = tsqrt((r - z.re) * 0.5f);
    bool pos = val(z.im) >= 0.0f;
    T ay = pos ? z.im : -z.im;
    return {ay / (t * 2.0f), pos ? t : -t};
}

// ------------------------------------------------------------------ Fresnel
// Reflection Mueller block in the s/p frames, [[A,B,0,0],[B,A,0,0],[0,0,C,S],[0,0,-S,C]]
// from r_s = (ei ci - et ct)/(ei ci + et ct), r_p = (et ci - ei ct)/(et ci + ei ct):
// A = (|rs|^2+|rp|^2)/2, B = (|rs|^2-|rp|^2)/2, C + iS = rs conj(rp).
template <class T> struct ABCS { T A, B, C, S; };
template <class T> __device__ __forceinline__ ABCS<T> fresnel_reflect(float cos_i, T eta_i, Cx<T> eta_t) {
    Cx<T> ei = {eta_i, T(0.0f)};
    Cx<T> q = cdiv(ei, eta_t);
    Cx<T> q2 = cmul(q, q);
    float sin2 = 1.0f - cos_i * cos_i;
    Cx<T> arg = {T(1.0f) - q2.re * sin2, -(q2.im * sin2)};
    Cx<T> ct = csqrt(arg);
    Cx<T> a = {eta_i * cos_i, T(0.0f)};
    Cx<T> b = cmul(eta_t, ct);
    Cx<T> rs = cdiv(Cx<T>{a.re - b.re, a.im - b.im}, Cx<T>{a.re + b.re, a.im + b.im});
    Cx<T> c = {eta_t.re * cos_i, eta_t.im * cos_i};
    Cx<T> d = {eta_i * ct.re, eta_i * ct.im};
    Cx<T> rp = cdiv(Cx<T>{c.re - d.re, c.im - d.im}, Cx<T>{c.re + d.re, c.im + d.im});
    T ns = rs.re * rs.re + rs.im * rs.im, np = rp.re * rp.re + rp.im * rp.im;
    return {(ns + np) * 0.5f, (ns - np) * 0.5f, rs.re * rp.re + rs.im * rp.im, rs.im * rp.re - rs.re * rp.im};
}
// real indices (dielectrics); total internal reflection handled by the complex path
template <class T> __device__ __forceinline__ ABCS<T> fresnel_reflect_real(float cos_i, T eta_i, T eta_t) {
    T q = eta_i / eta_t;
    T arg = T(1.0f) - q * q * (1.0f - cos_i * cos_i);
    if (val(arg) < 0.0f) return fresnel_reflect<T>(cos_i, eta_i, Cx<T>{eta_t, T(0.0f)});
    T ct = tsqrt(arg);
    T rs = (eta_i * cos_i - eta_t * ct) / (eta_i * cos_i + eta_t * ct);
    T rp = (eta_t * cos_i - eta_i * ct) / (eta_t * cos_i + eta_i * ct);
    return {(rs * rs + rp * rp) * 0.5f, (rs * rs - rp * rp) * 0.5f, rs * rp, T(0.0f)};
}
__device__ __forceinline__ float fresnel_unpolarized(float cos_i, float eta_i, float eta_t) {
    return fresnel_reflect_real<float>(cos_i, eta_i, eta_t).A;
}
// transmission of light from index eta_i into eta_t (no TIR), with the power
// factor eta_t cos_t / (eta_i cos_i)
template <class T> __device__ __forceinline__ ABCS<T> fresnel_transmit(float cos_i, T eta_i, T eta_t) {
    T q = eta_i / eta_t;
    T ct = tsqrt(T(1.0f) - q * q * (1.0f - cos_i * cos_i));
    T ts = (eta_i * cos_i * 2.0f) / (eta_i * cos_i + eta_t * ct);
    T tp = (eta_i * cos_i * 2.0f) / (eta_t * cos_i + eta_i * ct);
    T fac = (eta_t * ct) / (eta_i * cos_i);
    return {fac * (ts * ts + tp * tp) * 0.5f, fac * (ts * ts - tp * tp) * 0.5f, fac * ts * tp, T(0.0f)};
}

// ------------------------------------------------------------------ GGX (Walter et al. 2007)
// the cosines with the shading normal carry derivatives under a normal map: type C
// GGX normal distribution D(h) = a^2 / (pi k^2), k = (a^2 - 1) cos^2 + 1 = sin^2 + a^2 cos^2
// (Walter et al. 2007).  The caller passes sin^2 of the half vector's angle to the normal as
// |n x h|^2: near the lobe's peak 1 - cos^2 would cancel in FP32 (for a = 0.01 the peak's k
// is ~1e-4, and cos_h carries a rounding error of ~1e-7).
template <class T, class C = float> __device__ __forceinline__ T ggx_D(C cos_h, C sin2_h, T alpha) {
    if (val(cos_h) <= 0.0f) return T(0.0f);
    T a2 = alpha * alpha;
    T k = a2 * (cos_h * cos_h) + sin2_h;
    return a2 / (k * k * kPi);
}
template <class T, class C = float> __device__ __forceinline__ T ggx_G1(C cos_v, float cos_vh, T alpha) {
    if (cos_vh * val(cos_v) <= 0.0f) return T(0.0f);
    C t2 = (1.0f - cos_v * cos_v) / (cos_v * cos_v);
    return T(2.0f) / (tsqrt(alpha * alpha * t2 + 1.0f) + 1.0f);
}

}  // namespace dppt
