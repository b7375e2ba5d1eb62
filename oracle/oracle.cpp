// FP64 CPU oracle for differentiable polarized path tracing.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
// definition of what the GPU library computes; only the test-suite, the smoke
// check and the benchmark's CPU-baseline leg may load it.  It shares no code,
// header, table or helper with the CUDA library: every routine below was
// written separately from the paper's definitions.
//
// What it computes (Sec. 3 and Sec. 4 of the paper):
//   * the Monte Carlo estimate of the rendering equation (Eq. 2) for polarized
//     light: Stokes vectors carried through 4x4 Mueller operators (Sec. 3.3),
//     with reference-frame rotations before every product (Sec. 3.3,
//     "Coordinate Conventions");
//   * the reverse-mode derivative of that estimator with the sampling
//     decisions detached (Sec. 3.2 / PRB), by two independent routes:
//       mode 0  conventional taped AD over the whole path ("Conv. AD", Sec. 5.1);
//       mode 1  cached suffix replay (Sec. 4.3, Fig. 2): primal pass stores the
//               per-vertex emission E_i and transport factor W_i, a backward
//               fold builds the suffixes L[i] = E_i + W_i L[i+1], and the
//               adjoint walks the path forward with the prefix adjoint a,
//               differentiating only the local vertex (AD inside the loop
//               body only) and multiplying by the cached L[i+1] -- no inverse.
//   * a frozen-sampling estimator F(pi) (sampling from pi0, values from pi)
//     whose central differences check both derivative routes.
//
// Conventions that the paper leaves to its host renderer (Stokes frames and the
// rotation sign, the signs of the Fresnel blocks' C and S terms, the depth and
// MIS conventions) are fixed here and implemented again, independently, in the
// CUDA library.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ============================================================ Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of the 4x64
// Philox S-box with the published multipliers and Weyl key increments.
void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Eight uniforms in [0,1) for (path, vertex): 24-bit mantissas, exact in float and double.
struct Uniforms { double u[8]; };
Uniforms draw(uint64_t seed, uint64_t pass, uint64_t stream, uint64_t path, uint64_t vertex) {
    uint64_t key[2] = {seed ^ (pass * 0x9E3779B97F4A7C15ULL), stream};
    uint64_t ctr[4] = {path, vertex, 0, 0};
    uint64_t o[4];
    philox4x64_10(ctr, key, o);
    Uniforms r;
    for (int k = 0; k < 4; ++k) {
        uint32_t lo = (uint32_t)(o[k] & 0xffffffffULL), hi = (uint32_t)(o[k] >> 32);
        r.u[2 * k] = (double)(lo >> 8) * (1.0 / 16777216.0);
        r.u[2 * k + 1] = (double)(hi >> 8) * (1.0 / 16777216.0);
    }
    return r;
}

// ============================================================ taped reverse AD
// A Wengert list: every operation on a Var appends one node holding the local
// partial derivatives w.r.t. (at most) two operands.  Operand index >= 0 is a
// tape node, -1 a constant, <= -2 the parameter leaf (-2 - k).
struct TNode { int a, b; double da, db; };
thread_local std::vector<TNode> g_tape;
thread_local size_t g_tape_peak = 0;
thread_local double g_tape_total = 0;   // nodes of all whole-path tapes (conventional AD)

struct Var {
    double v; int i;
    Var() : v(0), i(-1) {}
    Var(double x) : v(x), i(-1) {}
    static Var leaf(double x, int64_t k) { Var r(x); r.i = (int)(-2 - k); return r; }
};
inline Var mk1(double v, const Var& a, double da) {
    if (a.i == -1) return Var(v);
    g_tape.push_back({a.i, -1, da, 0.0});
    Var r(v); r.i = (int)g_tape.size() - 1; return r;
}
inline Var mk2(double v, const Var& a, double da, const Var& b, double db) {
    if (a.i == -1 && b.i == -1) return Var(v);
    g_tape.push_back({a.i, b.i, da, db});
    Var r(v); r.i = (int)g_tape.size() - 1; return r;
}
inline Var operator+(const Var& a, const Var& b) { return mk2(a.v + b.v, a, 1.0, b, 1.0); }
inline Var operator-(const Var& a, const Var& b) { return mk2(a.v - b.v, a, 1.0, b, -1.0); }
inline Var operator*(const Var& a, const Var& b) { return mk2(a.v * b.v, a, b.v, b, a.v); }
inline Var operator/(const Var& a, const Var& b) { return mk2(a.v / b.v, a, 1.0 / b.v, b, -a.v / (b.v * b.v)); }
inline Var operator-(const Var& a) { return mk1(-a.v, a, -1.0); }
inline Var operator+(const Var& a, double b) { return mk1(a.v + b, a, 1.0); }
inline Var operator+(double a, const Var& b) { return mk1(a + b.v, b, 1.0); }
inline Var operator-(const Var& a, double b) { return mk1(a.v - b, a, 1.0); }
inline Var operator-(double a, const Var& b) { return mk1(a - b.v, b, -1.0); }
inline Var operator*(const Var& a, double b) { return mk1(a.v * b, a, b); }
inline Var operator*(double a, const Var& b) { return mk1(a * b.v, b, a); }
inline Var operator/(const Var& a, double b) { return mk1(a.v / b, a, 1.0 / b); }
inline Var operator/(double a, const Var& b) { return mk1(a / b.v, b, -a / (b.v * b.v)); }
inline Var& operator+=(Var& a, const Var& b) { a = a + b; return a; }
inline Var sqrt(const Var& a) { double s = std::sqrt(a.v); return mk1(s, a, 0.5 / s); }
inline Var sin(const Var& a) { return mk1(std::sin(a.v), a, std::cos(a.v)); }
inline Var cos(const Var& a) { return mk1(std::cos(a.v), a, -std::sin(a.v)); }
inline double val(const Var& a) { return a.v; }
using std::sqrt;
using std::sin;
using std::cos;
inline double val(double a) { return a; }

// Reverse sweep from `out` with seed `s`; leaf adjoints are added into grad[k].
void tape_backward(const Var& out, double s, double* grad) {
    g_tape_peak = std::max(g_tape_peak, g_tape.size());
    if (out.i <= -2) { grad[-2 - out.i] += s; return; }
    if (out.i < 0) return;
    std::vector<double> adj(g_tape.size(), 0.0);
    adj[out.i] = s;
    for (int n = (int)g_tape.size() - 1; n >= 0; --n) {
        double g = adj[n];
        if (g == 0.0) continue;
        const TNode& t = g_tape[n];
        if (t.a >= 0) adj[t.a] += g * t.da; else if (t.a <= -2) grad[-2 - t.a] += g * t.da;
        if (t.b >= 0) adj[t.b] += g * t.db; else if (t.b <= -2) grad[-2 - t.b] += g * t.db;
    }
}

// ============================================================ small math
struct V3 { double x, y, z; };
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator*(double s, V3 a) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double length(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return a * (1.0 / length(a)); }
inline V3 ld3(const double* p) { return {p[0], p[1], p[2]}; }
inline double axis(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// Orthonormal tangent of a unit vector n (Duff et al. 2017, "Building an
// Orthonormal Basis, Revisited", first vector); with t2 = n x t1 the triple
// (t1, t2, n) is right handed.  It is the reference x axis of the Stokes
// frame of light propagating along n.
inline V3 onb_t1(V3 n) {
    double sg = std::copysign(1.0, n.z);
    double a = -1.0 / (sg + n.z);
    double b = n.x * n.y * a;
    return {1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x};
}
inline V3 onb_t2(V3 n) {
    double sg = std::copysign(1.0, n.z);
    double a = -1.0 / (sg + n.z);
    double b = n.x * n.y * a;
    return {b, sg + n.y * n.y * a, -n.y};
}

template <class T> struct Cx { T re, im; };
template <class T> Cx<T> cadd(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> Cx<T> csub(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> Cx<T> cmul(Cx<T> a, Cx<T> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
template <class T> Cx<T> cscale(Cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> Cx<T> cdiv(Cx<T> a, Cx<T> b) {
    T d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <class T> T cnorm2(Cx<T> a) { return a.re * a.re + a.im * a.im; }
// Principal square root (branch cut on the negative real axis, Re >= 0), in a
// form with no cancellation; a purely negative real argument with +0
// imaginary part maps to +i sqrt(|x|).
template <class T> Cx<T> csqrt(Cx<T> z) {
    T r = sqrt(z.re * z.re + z.im * z.im);
    if (val(r) == 0.0) return {T(0.0), T(0.0)};
    if (val(z.re) >= 0.0) {
        T t = sqrt((r + z.re) * 0.5);
        return {t, z.im / (t * 2.0)};
    }
    T t = sqrt((r - z.re) * 0.5);
    T ay = val(z.im) >= 0.0 ? z.im : -z.im;
    T im = val(z.im) >= 0.0 ? t : -t;
    return {ay / (t * 2.0), im};
}

template <class T> struct M4 {
    T m[4][4];
    static M4 zero() { M4 r; for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) r.m[i][j] = T(0.0); return r; }
    static M4 ident() { M4 r = zero(); for (int i = 0; i < 4; ++i) r.m[i][i] = T(1.0); return r; }
};
template <class T, class U> M4<T> mmul(const M4<T>& a, const M4<U>& b) {
    M4<T> r;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            T s = a.m[i][0] * b.m[0][j];
            for (int k = 1; k < 4; ++k) s = s + a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}
template <class T> M4<T> mmul_dl(const M4<double>& a, const M4<T>& b) {
    M4<T> r;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            T s = a.m[i][0] * b.m[0][j];
            for (int k = 1; k < 4; ++k) s = s + a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}
template <class T> M4<T> mscale(const M4<T>& a, T s) {
    M4<T> r; for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) r.m[i][j] = a.m[i][j] * s; return r;
}
template <class T> M4<T> madd(const M4<T>& a, const M4<T>& b) {
    M4<T> r; for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j]; return r;
}
template <class T> M4<T> to_t(const M4<double>& a) {
    M4<T> r; for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) r.m[i][j] = T(a.m[i][j]); return r;
}
template <class T> struct S4 { T s[4]; };
template <class T> S4<T> szero() { S4<T> r; for (int i = 0; i < 4; ++i) r.s[i] = T(0.0); return r; }
template <class T, class U> S4<T> mvec(const M4<T>& a, const S4<U>& v) {
    S4<T> r;
    for (int i = 0; i < 4; ++i) {
        T s = a.m[i][0] * v.s[0];
        for (int k = 1; k < 4; ++k) s = s + a.m[i][k] * v.s[k];
        r.s[i] = s;
    }
    return r;
}

// Stokes rotator R: re-expresses a Stokes vector given in a frame whose x axis
// is x_from into the frame whose x axis is x_to, both perpendicular to the
// propagation direction p and with y = p x x.  With x_to = cos(phi) x_from +
// sin(phi) y_from, R = [[1,0,0,0],[0,c,s,0],[0,-s,c,0],[0,0,0,1]], c = cos 2phi,
// s = sin 2phi.  Inputs need not be unit length (c, s are normalised).
template <class T> M4<T> rot_cs(T c, T s) {
    M4<T> r = M4<T>::zero();
    r.m[0][0] = T(1.0); r.m[3][3] = T(1.0);
    r.m[1][1] = c; r.m[1][2] = s; r.m[2][1] = -s; r.m[2][2] = c;
    return r;
}
template <class T> M4<T> rot_frames(V3 p, V3 x_from, const T xt[3]) {
    V3 y_from = cross(p, x_from);
    T cf = xt[0] * x_from.x + xt[1] * x_from.y + xt[2] * x_from.z;
    T sf = xt[0] * y_from.x + xt[1] * y_from.y + xt[2] * y_from.z;
    T n2 = cf * cf + sf * sf;
    return rot_cs<T>((cf * cf - sf * sf) / n2, (cf * sf * 2.0) / n2);
}
// rotation out of a (possibly parameter-dependent) frame x_from into a fixed x_to
template <class T> M4<T> rot_frames_from(V3 p, const T xf[3], V3 x_to) {
    // y_from = p x x_from
    T yf[3] = {xf[2] * p.y - xf[1] * p.z, xf[0] * p.z - xf[2] * p.x, xf[1] * p.x - xf[0] * p.y};
    T cf = xf[0] * x_to.x + xf[1] * x_to.y + xf[2] * x_to.z;
    T sf = yf[0] * x_to.x + yf[1] * x_to.y + yf[2] * x_to.z;
    T n2 = cf * cf + sf * sf;
    return rot_cs<T>((cf * cf - sf * sf) / n2, (cf * sf * 2.0) / n2);
}
M4<double> rot_fixed(V3 p, V3 x_from, V3 x_to) {
    double xt[3] = {x_to.x, x_to.y, x_to.z};
    return rot_frames<double>(p, x_from, xt);
}

// Linear polarizer with transmission axis along the frame's x axis, and a
// linear retarder of retardance delta with fast axis along x (Collett 2005).
template <class T> M4<T> polarizer0() {
    M4<T> r = M4<T>::zero();
    r.m[0][0] = T(0.5); r.m[0][1] = T(0.5); r.m[1][0] = T(0.5); r.m[1][1] = T(0.5);
    return r;
}
template <class T> M4<T> retarder0(double delta) {
    M4<T> r = M4<T>::zero();
    r.m[0][0] = T(1.0); r.m[1][1] = T(1.0);
    r.m[2][2] = T(std::cos(delta)); r.m[2][3] = T(std::sin(delta));
    r.m[3][2] = T(-std::sin(delta)); r.m[3][3] = T(std::cos(delta));
    return r;
}
// Element rotated by theta in the sensor frame: R(-theta) M R(theta).
template <class T> M4<T> rotated_element(const M4<T>& m, T theta) {
    T c = cos(theta * 2.0), s = sin(theta * 2.0);
    return mmul(mmul(rot_cs<T>(c, -s), m), rot_cs<T>(c, s));
}

// Fresnel amplitude coefficients for light incident from a medium of real
// index eta_i at cos(theta_i) onto a medium of (possibly complex) index eta_t:
//   r_s = (eta_i cos_i - eta_t cos_t)/(eta_i cos_i + eta_t cos_t)
//   r_p = (eta_t cos_i - eta_i cos_t)/(eta_t cos_i + eta_i cos_t)
// with cos_t the principal root of 1 - (eta_i/eta_t)^2 sin^2_i (complex for
// conductors and total internal reflection).  The reflection Mueller matrix in
// the s/p frames is [[A,B,0,0],[B,A,0,0],[0,0,C,S],[0,0,-S,C]] with
// A = (|rs|^2+|rp|^2)/2, B = (|rs|^2-|rp|^2)/2, C = Re(rs rp*), S = Im(rs rp*).
template <class T> struct FresnelABCS { T A, B, C, S; };
template <class T> FresnelABCS<T> fresnel_reflect(double cos_i, T eta_i, Cx<T> eta_t) {
    Cx<T> ei = {eta_i, T(0.0)};
    Cx<T> ratio = cdiv(ei, eta_t);
    Cx<T> ratio2 = cmul(ratio, ratio);
    T sin2 = T(1.0 - cos_i * cos_i);
    Cx<T> one = {T(1.0), T(0.0)};
    Cx<T> cos_t = csqrt(csub(one, cscale(ratio2, sin2)));
    Cx<T> ci = {T(cos_i), T(0.0)};
    Cx<T> a = cmul(ei, ci), b = cmul(eta_t, cos_t);
    Cx<T> rs = cdiv(csub(a, b), cadd(a, b));
    Cx<T> c = cmul(eta_t, ci), d = cmul(ei, cos_t);
    Cx<T> rp = cdiv(csub(c, d), cadd(c, d));
    T ns = cnorm2(rs), np = cnorm2(rp);
    Cx<T> rsp = cmul(rs, Cx<T>{rp.re, -rp.im});
    return {(ns + np) * 0.5, (ns - np) * 0.5, rsp.re, rsp.im};
}
// Transmission (real indices, no total internal reflection): t_s, t_p with the
// power factor eta_t cos_t / (eta_i cos_i).
template <class T> FresnelABCS<T> fresnel_transmit(double cos_i, T eta_i, T eta_t) {
    T ratio = eta_i / eta_t;
    T cos_t = sqrt(T(1.0) - ratio * ratio * (1.0 - cos_i * cos_i));
    T ts = (eta_i * cos_i * 2.0) / (eta_i * cos_i + eta_t * cos_t);
    T tp = (eta_i * cos_i * 2.0) / (eta_t * cos_i + eta_i * cos_t);
    T fac = (eta_t * cos_t) / (eta_i * cos_i);
    return {fac * (ts * ts + tp * tp) * 0.5, fac * (ts * ts - tp * tp) * 0.5, fac * ts * tp, T(0.0)};
}
template <class T> M4<T> abcs_matrix(const FresnelABCS<T>& f) {
    M4<T> r = M4<T>::zero();
    r.m[0][0] = f.A; r.m[0][1] = f.B; r.m[1][0] = f.B; r.m[1][1] = f.A;
    r.m[2][2] = f.C; r.m[2][3] = f.S; r.m[3][2] = -f.S; r.m[3][3] = f.C;
    return r;
}
// unpolarized reflectance (A of the reflection matrix) for sampling decisions
double fresnel_unpolarized(double cos_i, double eta_i, double eta_t) {
    return fresnel_reflect<double>(cos_i, eta_i, Cx<double>{eta_t, 0.0}).A;
}

// GGX (Trowbridge-Reitz) distribution and separable Smith masking, Walter et
// al. 2007, with alpha = roughness (isotropic).
// The cosines with the shading normal may carry derivatives too (normal maps): type C.
template <class T, class C = double> T ggx_D(C cos_h, T alpha) {
    if (val(cos_h) <= 0.0) return T(0.0);
    T a2 = alpha * alpha;
    T k = (a2 - 1.0) * (cos_h * cos_h) + 1.0;
    return a2 / (k * k * M_PI);
}
template <class T, class C = double> T ggx_G1(C cos_v, double cos_vh, T alpha) {
    if (cos_vh * val(cos_v) <= 0.0) return T(0.0);
    C t2 = (1.0 - cos_v * cos_v) / (cos_v * cos_v);
    return T(2.0) / (sqrt(alpha * alpha * t2 + 1.0) + 1.0);
}

// ============================================================ scene
enum { MAT_DIFFUSE = 0, MAT_SMOOTH_DIELECTRIC = 1, MAT_CONDUCTOR_GGX = 2, MAT_PLASTIC_GGX = 3,
       MAT_POLARIZER_SHEET = 4, MAT_RETARDER_SHEET = 5, MAT_EMITTER = 6 };
enum { FILTER_NONE = 0, FILTER_POLARIZER = 1, FILTER_QWP_POLARIZER = 2 };

struct Mat {
    int type, albedo_tex, rough_tex, ior_index, sheet_index, normal_tex;
    double eta_re, eta_im, t1[3], t2[3], retard, emission;
};
struct Light { V3 o, e1, e2, n; double area; };
struct Tex { int64_t off, w, h, ch; };
struct Cam { V3 org, fwd, right, up; double tanh; };
struct BNode { double lo[3], hi[3]; int left, right, start, count; };

struct Stats { double rays, shadow_rays, vertices, nodes, tri_tests, sph_tests, paths; };
thread_local Stats g_stats;

struct Scene {
    std::vector<V3> v; std::vector<double> uv; std::vector<int> idx, tmat, tlight;
    std::vector<double> sph; std::vector<int> smat;
    std::vector<Mat> mats; std::vector<Light> lights; std::vector<Tex> tex; std::vector<Cam> cams;
    std::vector<BNode> nodes; std::vector<int> order;
    double eps;
    int F() const { return (int)tmat.size(); }
};

// median-split BVH over triangle centroids (the oracle's own structure)
void bvh_build(Scene& s) {
    int F = s.F();
    s.order.resize(F);
    for (int i = 0; i < F; ++i) s.order[i] = i;
    std::vector<V3> cen(F);
    std::vector<double> lo(3 * F), hi(3 * F);
    for (int i = 0; i < F; ++i) {
        V3 a = s.v[s.idx[3 * i]], b = s.v[s.idx[3 * i + 1]], c = s.v[s.idx[3 * i + 2]];
        cen[i] = (a + b + c) * (1.0 / 3.0);
        for (int k = 0; k < 3; ++k) {
            lo[3 * i + k] = std::min({axis(a, k), axis(b, k), axis(c, k)});
            hi[3 * i + k] = std::max({axis(a, k), axis(b, k), axis(c, k)});
        }
    }
    s.nodes.clear();
    if (F == 0) return;
    struct Job { int node, start, count; };
    s.nodes.push_back({});
    std::vector<Job> st = {{0, 0, F}};
    while (!st.empty()) {
        Job j = st.back(); st.pop_back();
        BNode n;
        for (int k = 0; k < 3; ++k) { n.lo[k] = 1e300; n.hi[k] = -1e300; }
        double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
        for (int i = j.start; i < j.start + j.count; ++i) {
            int t = s.order[i];
            for (int k = 0; k < 3; ++k) {
                n.lo[k] = std::min(n.lo[k], lo[3 * t + k]);
                n.hi[k] = std::max(n.hi[k], hi[3 * t + k]);
                clo[k] = std::min(clo[k], axis(cen[t], k));
                chi[k] = std::max(chi[k], axis(cen[t], k));
            }
        }
        n.start = j.start; n.count = j.count; n.left = n.right = -1;
        if (j.count > 4) {
            int ax = 0;
            for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
            int half = j.count / 2;
            std::nth_element(s.order.begin() + j.start, s.order.begin() + j.start + half,
                             s.order.begin() + j.start + j.count,
                             [&](int a, int b) { return axis(cen[a], ax) < axis(cen[b], ax); });
            n.left = (int)s.nodes.size(); s.nodes.push_back({});
            n.right = (int)s.nodes.size(); s.nodes.push_back({});
            st.push_back({n.left, j.start, half});
            st.push_back({n.right, j.start + half, j.count - half});
            n.count = 0;
        }
        s.nodes[j.node] = n;
    }
}

struct Ray { V3 o, d; };
struct Hit { double t; int prim; double b1, b2; };

bool slab(const BNode& n, const Ray& r, double tmax) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double o = axis(r.o, k), d = axis(r.d, k);
        if (d == 0.0) { if (o < n.lo[k] || o > n.hi[k]) return false; continue; }
        double a = (n.lo[k] - o) / d, b = (n.hi[k] - o) / d;
        if (a > b) std::swap(a, b);
        t0 = std::max(t0, a); t1 = std::min(t1, b);
        if (t0 > t1) return false;
    }
    return true;
}

// Moller-Trumbore ray/triangle test; returns t (or -1) and barycentrics.
double tri_hit(const Scene& s, int f, const Ray& r, double& b1, double& b2) {
    g_stats.tri_tests += 1;
    V3 p0 = s.v[s.idx[3 * f]], p1 = s.v[s.idx[3 * f + 1]], p2 = s.v[s.idx[3 * f + 2]];
    V3 e1 = p1 - p0, e2 = p2 - p0;
    V3 pv = cross(r.d, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return -1.0;
    double inv = 1.0 / det;
    V3 tv = r.o - p0;
    double u = dot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    V3 qv = cross(tv, e1);
    double w = dot(r.d, qv) * inv;
    if (w < 0.0 || u + w > 1.0) return -1.0;
    b1 = u; b2 = w;
    return dot(e2, qv) * inv;
}
// ray/sphere with the cancellation-free discriminant (r^2 - |l - (l.d) d|^2)
double sph_hit(const Scene& s, int k, const Ray& r, double tmax) {
    g_stats.sph_tests += 1;
    V3 c = ld3(&s.sph[4 * k]);
    double rad = s.sph[4 * k + 3];
    V3 l = r.o - c;
    double beta = dot(l, r.d);
    V3 f = l - r.d * beta;
    double disc = rad * rad - dot(f, f);
    if (disc < 0.0) return -1.0;
    double gam = dot(l, l) - rad * rad;
    double h = -beta - std::copysign(std::sqrt(disc), beta);
    if (h == 0.0) return -1.0;
    double ta = gam / h, tb = h;
    double t0 = std::min(ta, tb), t1 = std::max(ta, tb);
    if (t0 > 0.0 && t0 < tmax) return t0;
    if (t1 > 0.0 && t1 < tmax) return t1;
    return -1.0;
}

bool closest(const Scene& s, const Ray& r, Hit& h) {
    g_stats.rays += 1;
    h.t = 1e300; h.prim = -1;
    if (!s.nodes.empty()) {
        int stack[128]; int sp = 0; stack[sp++] = 0;
        while (sp) {
            const BNode& n = s.nodes[stack[--sp]];
            g_stats.nodes += 1;
            if (!slab(n, r, h.t)) continue;
            if (n.left < 0) {
                for (int i = n.start; i < n.start + n.count; ++i) {
                    int f = s.order[i];
                    double b1, b2;
                    double t = tri_hit(s, f, r, b1, b2);
                    if (t > 0.0 && (t < h.t || (t == h.t && f < h.prim))) { h.t = t; h.prim = f; h.b1 = b1; h.b2 = b2; }
                }
            } else { stack[sp++] = n.left; stack[sp++] = n.right; }
        }
    }
    for (int k = 0; k < (int)s.smat.size(); ++k) {
        double t = sph_hit(s, k, r, 1e300);
        int id = s.F() + k;
        if (t > 0.0 && (t < h.t || (t == h.t && id < h.prim))) { h.t = t; h.prim = id; }
    }
    return h.prim >= 0;
}

bool occluded(const Scene& s, const Ray& r, double tmax) {
    g_stats.shadow_rays += 1;
    if (!s.nodes.empty()) {
        int stack[128]; int sp = 0; stack[sp++] = 0;
        while (sp) {
            const BNode& n = s.nodes[stack[--sp]];
            g_stats.nodes += 1;
            if (!slab(n, r, tmax)) continue;
            if (n.left < 0) {
                for (int i = n.start; i < n.start + n.count; ++i) {
                    double b1, b2;
                    double t = tri_hit(s, s.order[i], r, b1, b2);
                    if (t > 0.0 && t < tmax) return true;
                }
            } else { stack[sp++] = n.left; stack[sp++] = n.right; }
        }
    }
    for (int k = 0; k < (int)s.smat.size(); ++k) {
        double t = sph_hit(s, k, r, tmax);
        if (t > 0.0 && t < tmax) return true;
    }
    return false;
}

// bilinear lookup with wrap addressing; texel centres at (i + 0.5) / w
struct TexTap { int64_t idx[4]; double w[4]; };
TexTap tex_taps(const Tex& t, double u, double v) {
    double x = u * (double)t.w - 0.5, y = v * (double)t.h - 0.5;
    double fx0 = std::floor(x), fy0 = std::floor(y);
    double fx = x - fx0, fy = y - fy0;
    int64_t x0 = (int64_t)fx0, y0 = (int64_t)fy0;
    auto wrap = [](int64_t a, int64_t n) { int64_t m = a % n; return m < 0 ? m + n : m; };
    int64_t xa = wrap(x0, t.w), xb = wrap(x0 + 1, t.w), ya = wrap(y0, t.h), yb = wrap(y0 + 1, t.h);
    TexTap tp;
    tp.idx[0] = t.off + (ya * t.w + xa) * t.ch; tp.w[0] = (1 - fx) * (1 - fy);
    tp.idx[1] = t.off + (ya * t.w + xb) * t.ch; tp.w[1] = fx * (1 - fy);
    tp.idx[2] = t.off + (yb * t.w + xa) * t.ch; tp.w[2] = (1 - fx) * fy;
    tp.idx[3] = t.off + (yb * t.w + xb) * t.ch; tp.w[3] = fx * fy;
    return tp;
}

// ============================================================ parameters
// Flat parameter vector: [tex | ior | le (L x 3 x 4) | sheet | theta (angles)].
struct Layout { int64_t tex, ior, le, sheet, theta, total; };

template <class T> struct Params {
    const double* p; Layout lay;
    T at(int64_t k) const;
};
template <> double Params<double>::at(int64_t k) const { return p[k]; }
template <> Var Params<Var>::at(int64_t k) const { return Var::leaf(p[k], k); }

template <class T> T tex_lookup(const Scene& s, const Params<T>& P, int tex, int ch, double u, double v) {
    const Tex& t = s.tex[tex];
    TexTap tp = tex_taps(t, u, v);
    int c = (int)std::min<int64_t>(ch, t.ch - 1);
    T r = P.at(P.lay.tex + tp.idx[0] + c) * tp.w[0];
    for (int k = 1; k < 4; ++k) r = r + P.at(P.lay.tex + tp.idx[k] + c) * tp.w[k];
    return r;
}

// Shading normal of a vertex with a normal map (a material's tangent-space map, three
// channels n_t = 2 c - 1 interpolated bilinearly): normalize(n_t.x T + n_t.y B + n_t.z N)
// with N the geometric normal on the side of wo, T the triangle's dP/du made normal to N
// and unit, B = N x T.  Without a normal map it is N.  Evaluated with parameters of type T
// so that the normal map's texels carry derivatives.
template <class T> struct N3 { T x, y, z; };
struct Vtx;
template <class T> N3<T> shading_normal(const Scene& s, const Params<T>& P, const Vtx& vt);

// ============================================================ path sampling
// One surface vertex of a sampled path.  Everything here is computed with the
// detached parameters pi0: directions, lobe and reflect/refract choices, pdfs
// and MIS weights.  The Mueller values are evaluated later from this record
// with the live parameters pi (T = double or Var).
struct Vtx {
    V3 x, ng, n, wo; double tu, tv; int prim, mat;
    V3 ngo, tan; bool nmap;   // geometric normal toward wo; normal map: tangent (unit, normal to ngo)
    bool emit_light; int light; double w_emit;
    bool nee; int nee_light; V3 wl; double nee_w;
    bool scatter; V3 wi; double pdf; int event; bool delta;
    double p_event; bool outside;
};

template <class T> N3<T> shading_normal(const Scene& s, const Params<T>& P, const Vtx& vt) {
    if (!vt.nmap) return {T(vt.n.x), T(vt.n.y), T(vt.n.z)};
    const Mat& m = s.mats[vt.mat];
    T a = tex_lookup<T>(s, P, m.normal_tex, 0, vt.tu, vt.tv) * 2.0 - 1.0;
    T b = tex_lookup<T>(s, P, m.normal_tex, 1, vt.tu, vt.tv) * 2.0 - 1.0;
    T c = tex_lookup<T>(s, P, m.normal_tex, 2, vt.tu, vt.tv) * 2.0 - 1.0;
    V3 N = vt.ngo, Tg = vt.tan, B = cross(N, Tg);
    T x = a * Tg.x + b * B.x + c * N.x;
    T y = a * Tg.y + b * B.y + c * N.y;
    T z = a * Tg.z + b * B.z + c * N.z;
    T l = sqrt(x * x + y * y + z * z);
    return {x / l, y / l, z / l};
}

struct Path {
    std::vector<Vtx> vs;
    V3 d1;        // camera ray direction
    uint32_t sig; // FNV-1a of (prim, event, nee) per vertex
};

double bsdf_pdf(const Scene& s, const Params<double>& P0, const Vtx& vt, V3 wi);

inline uint32_t fnv(uint32_t h, uint32_t x) {
    for (int k = 0; k < 4; ++k) { h ^= (x >> (8 * k)) & 0xff; h *= 16777619u; }
    return h;
}

double alpha_of(const Scene& s, const Params<double>& P0, const Vtx& vt) {
    const Mat& m = s.mats[vt.mat];
    return tex_lookup<double>(s, P0, m.rough_tex, 0, vt.tu, vt.tv);
}
double mean_albedo(const Scene& s, const Params<double>& P0, const Vtx& vt) {
    const Mat& m = s.mats[vt.mat];
    if (m.albedo_tex < 0) return 1.0;
    double a = 0;
    for (int c = 0; c < 3; ++c) a += tex_lookup<double>(s, P0, m.albedo_tex, c, vt.tu, vt.tv);
    return a / 3.0;
}
// probability of sampling the specular lobe of the rough dielectric pBRDF
double plastic_pspec(const Scene& s, const Params<double>& P0, const Vtx& vt) {
    const Mat& m = s.mats[vt.mat];
    double eta = P0.at(P0.lay.ior + m.ior_index);
    double fs = fresnel_unpolarized(dot(vt.wo, vt.n), 1.0, eta);
    double fd = mean_albedo(s, P0, vt);
    double tot = fs + fd;
    return tot > 0.0 ? fs / tot : 0.5;
}
double ggx_pdf(double alpha, V3 n, V3 wo, V3 wi) {
    V3 h = normalize(wo + wi);
    double ch = dot(h, n), oh = dot(wo, h);
    if (ch <= 0.0 || oh <= 0.0) return 0.0;
    return ggx_D<double>(ch, alpha) * ch / (4.0 * oh);
}
double bsdf_pdf(const Scene& s, const Params<double>& P0, const Vtx& vt, V3 wi) {
    const Mat& m = s.mats[vt.mat];
    double ci = dot(wi, vt.n);
    if (ci <= 0.0) return 0.0;
    if (m.type == MAT_DIFFUSE) return ci / M_PI;
    if (m.type == MAT_CONDUCTOR_GGX) return ggx_pdf(alpha_of(s, P0, vt), vt.n, vt.wo, wi);
    if (m.type == MAT_PLASTIC_GGX) {
        double ps = plastic_pspec(s, P0, vt);
        return ps * ggx_pdf(alpha_of(s, P0, vt), vt.n, vt.wo, wi) + (1.0 - ps) * ci / M_PI;
    }
    return 0.0;
}

struct JobDesc {
    int cam, W, H, spp, depth; uint64_t seed, pass, stream; int filter, nang;
};

V3 camera_dir(const Cam& c, int W, int H, int px, int py, double ju, double jv) {
    double aspect = (double)W / (double)H;
    double sx = (2.0 * (px + ju) / W - 1.0) * c.tanh * aspect;
    double sy = (1.0 - 2.0 * (py + jv) / H) * c.tanh;
    return normalize(c.fwd + c.right * sx + c.up * sy);
}

Path sample_path(const Scene& s, const Params<double>& P0, const JobDesc& J, int64_t pixel, int64_t sample) {
    Path path;
    uint32_t sig = 2166136261u;
    uint64_t pid = (uint64_t)(pixel * J.spp + sample);
    const Cam& cam = s.cams[J.cam];
    int px = (int)(pixel % J.W), py = (int)(pixel / J.W);
    Uniforms u0 = draw(J.seed, J.pass, J.stream, pid, 0);
    V3 d = camera_dir(cam, J.W, J.H, px, py, u0.u[0], u0.u[1]);
    path.d1 = d;
    Ray ray{cam.org, d};
    V3 xprev = cam.org;
    bool prev_delta = true;
    double prev_pdf = 0.0;
    int nL = (int)s.lights.size();
    g_stats.paths += 1;
    for (int v = 1; v <= J.depth; ++v) {
        Hit h;
        if (!closest(s, ray, h)) break;
        g_stats.vertices += 1;
        Vtx vt{};
        vt.prim = h.prim;
        vt.x = ray.o + ray.d * h.t;
        vt.wo = -ray.d;
        if (h.prim < s.F()) {
            int f = h.prim;
            V3 p0 = s.v[s.idx[3 * f]], p1 = s.v[s.idx[3 * f + 1]], p2 = s.v[s.idx[3 * f + 2]];
            vt.ng = normalize(cross(p1 - p0, p2 - p0));
            vt.mat = s.tmat[f];
            double w0 = 1.0 - h.b1 - h.b2;
            int i0 = s.idx[3 * f], i1 = s.idx[3 * f + 1], i2 = s.idx[3 * f + 2];
            vt.tu = w0 * s.uv[2 * i0] + h.b1 * s.uv[2 * i1] + h.b2 * s.uv[2 * i2];
            vt.tv = w0 * s.uv[2 * i0 + 1] + h.b1 * s.uv[2 * i1 + 1] + h.b2 * s.uv[2 * i2 + 1];
            vt.light = s.tlight[f];
        } else {
            int k = h.prim - s.F();
            V3 c = ld3(&s.sph[4 * k]);
            vt.ng = (vt.x - c) * (1.0 / s.sph[4 * k + 3]);
            vt.mat = s.smat[k];
            vt.tu = std::atan2(vt.ng.z, vt.ng.x) / (2.0 * M_PI) + 0.5;
            vt.tv = std::acos(std::max(-1.0, std::min(1.0, vt.ng.y))) / M_PI;
            vt.light = -1;
        }
        vt.n = dot(vt.ng, vt.wo) >= 0.0 ? vt.ng : -vt.ng;
        const Mat& m = s.mats[vt.mat];
        vt.ngo = vt.n;
        vt.nmap = false;
        if (m.normal_tex >= 0 && h.prim < s.F()) {
            // tangent of the triangle's (u, v) parametrization: dP/du
            int f = h.prim, i0 = s.idx[3 * f], i1 = s.idx[3 * f + 1], i2 = s.idx[3 * f + 2];
            V3 dp1 = s.v[i1] - s.v[i0], dp2 = s.v[i2] - s.v[i0];
            double du1 = s.uv[2 * i1] - s.uv[2 * i0], dv1 = s.uv[2 * i1 + 1] - s.uv[2 * i0 + 1];
            double du2 = s.uv[2 * i2] - s.uv[2 * i0], dv2 = s.uv[2 * i2 + 1] - s.uv[2 * i0 + 1];
            double r = du1 * dv2 - du2 * dv1;
            if (std::fabs(r) > 1e-20) {
                V3 t = (dp1 * dv2 - dp2 * dv1) * (1.0 / r);
                t = t - vt.ngo * dot(vt.ngo, t);
                double tl = length(t);
                if (tl > 1e-12) {
                    vt.tan = t * (1.0 / tl);
                    vt.nmap = true;
                    N3<double> ns = shading_normal<double>(s, P0, vt);
                    vt.n = V3{ns.x, ns.y, ns.z};
                }
            }
        }
        // emission reached by BSDF sampling (MIS against light sampling)
        if (vt.light >= 0) {
            const Light& L = s.lights[vt.light];
            double cl = dot(L.n, vt.wo);
            if (cl > 0.0) {
                vt.emit_light = true;
                if (prev_delta) vt.w_emit = 1.0;
                else {
                    double dist2 = dot(vt.x - xprev, vt.x - xprev);
                    double pl = dist2 / (cl * L.area * nL);
                    vt.w_emit = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
                }
            }
        }
        uint32_t ev = 0, neeflag = 2;
        if (m.type == MAT_EMITTER || v == J.depth) {
            vt.scatter = false;
            sig = fnv(fnv(fnv(sig, (uint32_t)vt.prim), ev), neeflag);
            path.vs.push_back(vt);
            break;
        }
        Uniforms U = draw(J.seed, J.pass, J.stream, pid, (uint64_t)v);
        bool delta = (m.type == MAT_SMOOTH_DIELECTRIC || m.type == MAT_POLARIZER_SHEET || m.type == MAT_RETARDER_SHEET);
        vt.delta = delta;
        // next-event estimation at non-delta vertices
        if (!delta && nL > 0) {
            int l = std::min((int)(U.u[4] * nL), nL - 1);
            const Light& L = s.lights[l];
            V3 y = L.o + L.e1 * U.u[5] + L.e2 * U.u[6];
            V3 dv = y - vt.x;
            double dist2 = dot(dv, dv), dist = std::sqrt(dist2);
            V3 wl = dv * (1.0 / dist);
            double cl = -dot(L.n, wl), cx = dot(vt.n, wl);
            neeflag = 0;
            if (cl > 0.0 && cx > 0.0 && dot(vt.ngo, wl) > 0.0) {
                V3 o2 = vt.x + vt.ngo * s.eps;
                V3 dd = y - o2;
                double dl = length(dd);
                if (!occluded(s, Ray{o2, dd * (1.0 / dl)}, dl * (1.0 - 1e-4))) {
                    double pl = dist2 / (cl * L.area * nL);
                    double pb = bsdf_pdf(s, P0, vt, wl);
                    double wmis = pl * pl / (pl * pl + pb * pb);
                    vt.nee = true; vt.nee_light = l; vt.wl = wl;
                    vt.nee_w = cx / pl * wmis;
                    neeflag = 1;
                }
            }
        }
        // BSDF sampling
        bool ok = true;
        V3 wi{0, 0, 0};
        if (m.type == MAT_DIFFUSE || (m.type == MAT_PLASTIC_GGX) || m.type == MAT_CONDUCTOR_GGX) {
            bool spec = m.type == MAT_CONDUCTOR_GGX;
            if (m.type == MAT_PLASTIC_GGX) { spec = U.u[0] < plastic_pspec(s, P0, vt); ev = spec ? 1 : 2; }
            V3 t1 = onb_t1(vt.n), t2 = onb_t2(vt.n);
            if (!spec) {
                double r = std::sqrt(U.u[1]), ph = 2.0 * M_PI * U.u[2];
                double lx = r * std::cos(ph), ly = r * std::sin(ph), lz = std::sqrt(std::max(0.0, 1.0 - U.u[1]));
                wi = t1 * lx + t2 * ly + vt.n * lz;
            } else {
                double al = alpha_of(s, P0, vt);
                double tan2 = al * al * U.u[1] / (1.0 - U.u[1]);
                double ch = 1.0 / std::sqrt(1.0 + tan2);
                double sh = std::sqrt(std::max(0.0, 1.0 - ch * ch));
                double ph = 2.0 * M_PI * U.u[2];
                V3 hv = t1 * (sh * std::cos(ph)) + t2 * (sh * std::sin(ph)) + vt.n * ch;
                double oh = dot(vt.wo, hv);
                if (oh <= 0.0) ok = false;
                else wi = hv * (2.0 * oh) - vt.wo;
            }
            if (ok && (dot(wi, vt.n) <= 0.0 || dot(wi, vt.ngo) <= 0.0)) ok = false;
            if (ok) { vt.pdf = bsdf_pdf(s, P0, vt, wi); if (!(vt.pdf > 0.0)) ok = false; }
        } else if (m.type == MAT_SMOOTH_DIELECTRIC) {
            double eta = P0.at(P0.lay.ior + m.ior_index);
            double co = dot(vt.wo, vt.ng);
            vt.outside = co > 0.0;
            double eo = vt.outside ? 1.0 : eta, et = vt.outside ? eta : 1.0;
            double c = std::fabs(co);
            double F = fresnel_unpolarized(c, eo, et);
            double r = eo / et, s2 = r * r * (1.0 - c * c);
            if (s2 >= 1.0) F = 1.0;
            if (U.u[0] < F) {
                ev = 1; vt.p_event = F;
                wi = vt.n * (2.0 * c) - vt.wo;
            } else {
                ev = 2; vt.p_event = 1.0 - F;
                double ct = std::sqrt(1.0 - s2);
                wi = -vt.wo * r + vt.n * (r * c - ct);
            }
            vt.pdf = 1.0;
        } else {  // sheets: straight pass-through
            wi = -vt.wo;
            vt.pdf = 1.0;
        }
        vt.event = (int)ev;
        sig = fnv(fnv(fnv(sig, (uint32_t)vt.prim), ev), neeflag);
        if (!ok) { vt.scatter = false; path.vs.push_back(vt); break; }
        vt.scatter = true; vt.wi = wi;
        path.vs.push_back(vt);
        double side = dot(wi, vt.ng) >= 0.0 ? 1.0 : -1.0;
        xprev = vt.x;
        ray = Ray{vt.x + vt.ng * (side * s.eps), wi};
        prev_delta = delta;
        prev_pdf = vt.pdf;
    }
    path.sig = fnv(sig, (uint32_t)path.vs.size());
    return path;
}

// ============================================================ evaluation
// E_v (emission reaching vertex v, in the Stokes frame of light leaving toward
// the previous vertex) and W_v (maps the frame of light arriving along -wi to
// that outgoing frame), per RGB channel, evaluated with parameters of type T.
template <class T> struct VEval { S4<T> E[3]; M4<T> W[3]; };

template <class T> S4<T> light_le(const Scene& s, const Params<T>& P, int l, int c) {
    S4<T> r;
    for (int k = 0; k < 4; ++k) r.s[k] = P.at(P.lay.le + 12 * l + 4 * c + k);
    (void)s;
    return r;
}
// frame rotation from the emitter frame (x = e1 projected) into the canonical frame of p
M4<double> emitter_rot(const Light& L, V3 p) {
    V3 xe = L.e1 - p * dot(L.e1, p);
    return rot_fixed(p, xe, onb_t1(p));
}

// reflection-type pBRDF value f(wo, wi) (without the cosine), per channel
template <class T> void bsdf_eval(const Scene& s, const Params<T>& P, const Vtx& vt, V3 wi, M4<T> f[3]) {
    const Mat& m = s.mats[vt.mat];
    for (int c = 0; c < 3; ++c) f[c] = M4<T>::zero();
    const N3<T> n = shading_normal<T>(s, P, vt);
    T ci = n.x * wi.x + n.y * wi.y + n.z * wi.z, co = n.x * vt.wo.x + n.y * vt.wo.y + n.z * vt.wo.z;
    if (val(ci) <= 0.0 || val(co) <= 0.0) return;
    T alb[3];
    for (int c = 0; c < 3; ++c) alb[c] = m.albedo_tex >= 0 ? tex_lookup<T>(s, P, m.albedo_tex, c, vt.tu, vt.tv) : T(1.0);
    if (m.type == MAT_DIFFUSE) {
        for (int c = 0; c < 3; ++c) f[c].m[0][0] = alb[c] * (1.0 / M_PI);
        return;
    }
    // specular microfacet lobe: D G F(h) / (4 cos_o cos_i) with frame rotations
    V3 h = normalize(vt.wo + wi);
    T ch = n.x * h.x + n.y * h.y + n.z * h.z;
    double oh = dot(vt.wo, h), ih = dot(wi, h);
    T al = tex_lookup<T>(s, P, m.rough_tex, 0, vt.tu, vt.tv);
    T DG = ggx_D<T, T>(ch, al) * ggx_G1<T, T>(co, oh, al) * ggx_G1<T, T>(ci, ih, al);
    T k = DG / (co * ci * 4.0);
    FresnelABCS<T> F;
    if (m.type == MAT_CONDUCTOR_GGX) F = fresnel_reflect<T>(ih, T(1.0), Cx<T>{T(m.eta_re), T(m.eta_im)});
    else F = fresnel_reflect<T>(ih, T(1.0), Cx<T>{P.at(P.lay.ior + m.ior_index), T(0.0)});
    V3 sx = cross(vt.wo, h);
    double sl = length(sx);
    V3 sax = sl > 1e-12 ? sx * (1.0 / sl) : onb_t1(vt.wo);
    M4<double> Rin = rot_fixed(-wi, onb_t1(-wi), sax);
    M4<double> Rout = rot_fixed(vt.wo, sax, onb_t1(vt.wo));
    M4<T> Ms = mmul_dl(Rout, mmul(abcs_matrix(F), to_t<T>(Rin)));
    for (int c = 0; c < 3; ++c) {
        T kc = m.type == MAT_CONDUCTOR_GGX ? k * alb[c] : k;
        f[c] = mscale(Ms, kc);
        if (m.type == MAT_PLASTIC_GGX) f[c].m[0][0] = f[c].m[0][0] + alb[c] * (1.0 / M_PI);
    }
}

template <class T> void sheet_axis(const Scene& s, const Params<T>& P, const Mat& m, V3 p, T xf[3]) {
    T th = P.at(P.lay.sheet + m.sheet_index);
    T ct = cos(th), st = sin(th);
    T t[3] = {ct * m.t1[0] + st * m.t2[0], ct * m.t1[1] + st * m.t2[1], ct * m.t1[2] + st * m.t2[2]};
    T tp = t[0] * p.x + t[1] * p.y + t[2] * p.z;
    xf[0] = t[0] - tp * p.x; xf[1] = t[1] - tp * p.y; xf[2] = t[2] - tp * p.z;
    (void)s;
}

template <class T> VEval<T> eval_vertex(const Scene& s, const Params<T>& P, const Vtx& vt) {
    VEval<T> r;
    for (int c = 0; c < 3; ++c) { r.E[c] = szero<T>(); r.W[c] = M4<T>::zero(); }
    const Mat& m = s.mats[vt.mat];
    if (vt.emit_light) {
        const Light& L = s.lights[vt.light];
        M4<double> R = emitter_rot(L, vt.wo);
        for (int c = 0; c < 3; ++c) {
            S4<T> le = light_le(s, P, vt.light, c);
            S4<T> e;
            for (int i = 0; i < 4; ++i) {
                T a = le.s[0] * R.m[i][0];
                for (int k = 1; k < 4; ++k) a = a + le.s[k] * R.m[i][k];
                e.s[i] = a * vt.w_emit;
            }
            r.E[c] = e;
        }
    }
    if (m.emission > 0.0)
        for (int c = 0; c < 3; ++c) r.E[c].s[0] = r.E[c].s[0] + m.emission;
    if (vt.nee) {
        const Light& L = s.lights[vt.nee_light];
        M4<double> R = emitter_rot(L, -vt.wl);
        M4<T> f[3];
        bsdf_eval<T>(s, P, vt, vt.wl, f);
        // nee_w holds the cosine with the detached shading normal: a normal map makes it live
        T wn = T(vt.nee_w);
        if (vt.nmap) {
            const N3<T> n = shading_normal<T>(s, P, vt);
            wn = (n.x * vt.wl.x + n.y * vt.wl.y + n.z * vt.wl.z) * (vt.nee_w / dot(vt.n, vt.wl));
        }
        for (int c = 0; c < 3; ++c) {
            S4<T> le = light_le(s, P, vt.nee_light, c);
            S4<T> lr = mvec(to_t<T>(R), le);
            S4<T> e = mvec(f[c], lr);
            for (int i = 0; i < 4; ++i) r.E[c].s[i] = r.E[c].s[i] + e.s[i] * wn;
        }
    }
    if (!vt.scatter) return r;
    V3 wi = vt.wi;
    if (m.type == MAT_DIFFUSE || m.type == MAT_CONDUCTOR_GGX || m.type == MAT_PLASTIC_GGX) {
        M4<T> f[3];
        bsdf_eval<T>(s, P, vt, wi, f);
        const N3<T> n = shading_normal<T>(s, P, vt);
        T w = (n.x * wi.x + n.y * wi.y + n.z * wi.z) * (1.0 / vt.pdf);
        for (int c = 0; c < 3; ++c) r.W[c] = mscale(f[c], w);
    } else if (m.type == MAT_SMOOTH_DIELECTRIC) {
        T eta = P.at(P.lay.ior + m.ior_index);
        T eo = vt.outside ? T(1.0) : eta, et = vt.outside ? eta : T(1.0);
        double c = dot(vt.wo, vt.n);
        V3 sx = cross(vt.wo, vt.n);
        double sl = length(sx);
        V3 sax = sl > 1e-12 ? sx * (1.0 / sl) : onb_t1(vt.wo);
        M4<double> Rin = rot_fixed(-wi, onb_t1(-wi), sax);
        M4<double> Rout = rot_fixed(vt.wo, sax, onb_t1(vt.wo));
        M4<T> M;
        if (vt.event == 1) {
            M = abcs_matrix(fresnel_reflect<T>(c, eo, Cx<T>{et, T(0.0)}));
            M = mscale(M, T(1.0 / vt.p_event));
        } else {
            // light travels from the wi side (index et) into the wo side (index eo)
            double ci = std::fabs(dot(wi, vt.n));
            M = abcs_matrix(fresnel_transmit<T>(ci, et, eo));
            T sc = (eo / et) * (eo / et);
            M = mscale(M, sc * (1.0 / vt.p_event));
        }
        M4<T> W = mmul_dl(Rout, mmul(M, to_t<T>(Rin)));
        for (int cc = 0; cc < 3; ++cc) r.W[cc] = W;
    } else if (m.type == MAT_POLARIZER_SHEET || m.type == MAT_RETARDER_SHEET) {
        V3 p = vt.wo;   // propagation direction is unchanged by the sheet
        T xf[3];
        sheet_axis(s, P, m, p, xf);
        M4<T> Rin = rot_frames<T>(p, onb_t1(p), xf);
        M4<T> Rout = rot_frames_from<T>(p, xf, onb_t1(p));
        M4<T> M = m.type == MAT_POLARIZER_SHEET ? polarizer0<T>() : retarder0<T>(m.retard);
        M4<T> W = mmul(Rout, mmul(M, Rin));
        for (int cc = 0; cc < 3; ++cc) r.W[cc] = W;
    }
    return r;
}

// camera: rotation of the path's first frame into the sensor frame, and the filter
M4<double> camera_rot(const Scene& s, int cam, V3 d1) {
    V3 p = -d1;
    V3 xr = s.cams[cam].right;
    V3 xs = xr - p * dot(xr, p);
    return rot_fixed(p, onb_t1(p), xs);
}
template <class T> M4<T> camera_filter(int filter, T theta) {
    if (filter == FILTER_NONE) return M4<T>::ident();
    M4<T> P = rotated_element<T>(polarizer0<T>(), theta);
    if (filter == FILTER_POLARIZER) return P;
    return mmul(P, retarder0<T>(M_PI / 2));
}

}  // namespace

// ============================================================ C interface
extern "C" {

void* orc_scene_create(int64_t nv, const double* verts, const double* uvs, int64_t nf, const int32_t* tris,
                       const int32_t* tri_mat, const int32_t* tri_light, int64_t ns, const double* spheres,
                       const int32_t* sph_mat, int64_t nm, const int32_t* mat_i /*nm x 6*/,
                       const double* mat_f /*nm x 10*/, int64_t nl, const double* lights /*nl x 9*/,
                       int64_t nt, const int64_t* tex_desc /*nt x 4*/, int64_t nc, const double* cams /*nc x 10*/,
                       double eps) {
    Scene* s = new Scene();
    s->v.resize(nv);
    for (int64_t i = 0; i < nv; ++i) s->v[i] = ld3(verts + 3 * i);
    s->uv.assign(uvs, uvs + 2 * nv);
    s->idx.assign(tris, tris + 3 * nf);
    s->tmat.assign(tri_mat, tri_mat + nf);
    s->tlight.assign(tri_light, tri_light + nf);
    s->sph.assign(spheres, spheres + 4 * ns);
    s->smat.assign(sph_mat, sph_mat + ns);
    for (int64_t i = 0; i < nm; ++i) {
        Mat m;
        m.type = mat_i[6 * i]; m.albedo_tex = mat_i[6 * i + 1]; m.rough_tex = mat_i[6 * i + 2];
        m.ior_index = mat_i[6 * i + 3]; m.sheet_index = mat_i[6 * i + 4]; m.normal_tex = mat_i[6 * i + 5];
        const double* f = mat_f + 10 * i;
        m.eta_re = f[0]; m.eta_im = f[1];
        m.t1[0] = f[2]; m.t1[1] = f[3]; m.t1[2] = f[4];
        m.t2[0] = f[5]; m.t2[1] = f[6]; m.t2[2] = f[7];
        m.retard = f[8]; m.emission = f[9];
        s->mats.push_back(m);
    }
    for (int64_t i = 0; i < nl; ++i) {
        Light L;
        L.o = ld3(lights + 9 * i); L.e1 = ld3(lights + 9 * i + 3); L.e2 = ld3(lights + 9 * i + 6);
        V3 c = cross(L.e1, L.e2);
        L.area = length(c); L.n = c * (1.0 / L.area);
        s->lights.push_back(L);
    }
    for (int64_t i = 0; i < nt; ++i) s->tex.push_back({tex_desc[4 * i], tex_desc[4 * i + 1], tex_desc[4 * i + 2], tex_desc[4 * i + 3]});
    for (int64_t i = 0; i < nc; ++i) {
        const double* c = cams + 10 * i;
        Cam cm;
        cm.org = ld3(c);
        cm.fwd = normalize(ld3(c + 3) - cm.org);
        cm.right = normalize(cross(cm.fwd, ld3(c + 6)));
        cm.up = cross(cm.right, cm.fwd);
        cm.tanh = std::tan(0.5 * c[9] * M_PI / 180.0);
        s->cams.push_back(cm);
    }
    s->eps = eps;
    bvh_build(*s);
    return s;
}

void orc_scene_destroy(void* sc) { delete (Scene*)sc; }

static JobDesc job_from(const int64_t* j) {
    JobDesc J;
    J.cam = (int)j[0]; J.W = (int)j[1]; J.H = (int)j[2]; J.spp = (int)j[3]; J.depth = (int)j[4];
    J.seed = (uint64_t)j[5]; J.pass = (uint64_t)j[6]; J.stream = (uint64_t)j[7];
    J.filter = (int)j[8]; J.nang = (int)j[9];
    return J;
}
static Layout layout_from(const int64_t* l) { return {l[0], l[1], l[2], l[3], l[4], l[5]}; }

// Primal render of the listed pixels.  Sampling uses P0 (detached), values use
// P; with P == P0 this is the plain estimator.  out: [angles][npix][3][4];
// path_out (nullable): raw sensor-frame Stokes per path [npix*spp][3][4];
// path_sig (nullable): signature per path.
int orc_render(void* sc, const int64_t* job, const int64_t* pixels, int64_t npix, const double* P0,
               const double* Pv, const int64_t* layout, double* out, double* path_out, uint32_t* path_sig) {
    const Scene& s = *(const Scene*)sc;
    JobDesc J = job_from(job);
    Layout lay = layout_from(layout);
    Params<double> p0{P0, lay}, pv{Pv, lay};
    int A = J.filter == FILTER_NONE ? 1 : J.nang;
    std::vector<M4<double>> C(A);
    for (int a = 0; a < A; ++a) C[a] = camera_filter<double>(J.filter, J.filter == FILTER_NONE ? 0.0 : Pv[lay.theta + a]);
    for (int64_t ip = 0; ip < npix; ++ip) {
        int64_t pix = pixels[ip];
        double acc[3][4] = {};
        for (int smp = 0; smp < J.spp; ++smp) {
            Path path = sample_path(s, p0, J, pix, smp);
            int n = (int)path.vs.size();
            S4<double> L[3];
            for (int c = 0; c < 3; ++c) L[c] = szero<double>();
            for (int v = n - 1; v >= 0; --v) {   // backward fold L = E + W L
                VEval<double> e = eval_vertex<double>(s, pv, path.vs[v]);
                for (int c = 0; c < 3; ++c) {
                    S4<double> wl = mvec(e.W[c], L[c]);
                    for (int k = 0; k < 4; ++k) L[c].s[k] = e.E[c].s[k] + wl.s[k];
                }
            }
            M4<double> Rc = camera_rot(s, J.cam, path.d1);
            int64_t prow = ip * J.spp + smp;
            for (int c = 0; c < 3; ++c) {
                S4<double> raw = mvec(Rc, L[c]);
                for (int k = 0; k < 4; ++k) acc[c][k] += raw.s[k];
                if (path_out) for (int k = 0; k < 4; ++k) path_out[(prow * 3 + c) * 4 + k] = raw.s[k];
            }
            if (path_sig) path_sig[prow] = path.sig;
        }
        for (int a = 0; a < A; ++a)
            for (int c = 0; c < 3; ++c) {
                S4<double> raw;
                for (int k = 0; k < 4; ++k) raw.s[k] = acc[c][k] / J.spp;
                S4<double> o = mvec(C[a], raw);
                for (int k = 0; k < 4; ++k) out[((a * npix + ip) * 3 + c) * 4 + k] = o.s[k];
            }
    }
    return 0;
}

// Reverse-mode gradient of sum_{a,pix,c,k} dI[a][pix][c][k] * I[a][pix][c][k]
// over the listed pixels.  mode 0: conventional taped AD of the whole path;
// mode 1: cached suffix replay.  grad (flat, same layout as P) is accumulated.
int orc_gradient(void* sc, const int64_t* job, const int64_t* pixels, int64_t npix, const double* Pd,
                 const int64_t* layout, const double* dI, double* grad, int mode) {
    const Scene& s = *(const Scene*)sc;
    JobDesc J = job_from(job);
    Layout lay = layout_from(layout);
    Params<double> pd{Pd, lay};
    Params<Var> pvar{Pd, lay};
    int A = J.filter == FILTER_NONE ? 1 : J.nang;
    for (int64_t ip = 0; ip < npix; ++ip) {
        int64_t pix = pixels[ip];
        for (int smp = 0; smp < J.spp; ++smp) {
            Path path = sample_path(s, pd, J, pix, smp);
            int n = (int)path.vs.size();
            M4<double> Rc = camera_rot(s, J.cam, path.d1);
            const double inv_spp = 1.0 / J.spp;
            if (mode == 0) {
                // ---- conventional AD: the whole path on one tape
                g_tape.clear();
                S4<Var> L[3];
                for (int c = 0; c < 3; ++c) L[c] = szero<Var>();
                for (int v = n - 1; v >= 0; --v) {
                    VEval<Var> e = eval_vertex<Var>(s, pvar, path.vs[v]);
                    for (int c = 0; c < 3; ++c) {
                        S4<Var> wl = mvec(e.W[c], L[c]);
                        for (int k = 0; k < 4; ++k) L[c].s[k] = e.E[c].s[k] + wl.s[k];
                    }
                }
                Var J0(0.0);
                for (int a = 0; a < A; ++a) {
                    Var th = J.filter == FILTER_NONE ? Var(0.0) : pvar.at(lay.theta + a);
                    M4<Var> CR = mmul(camera_filter<Var>(J.filter, th), to_t<Var>(Rc));
                    for (int c = 0; c < 3; ++c) {
                        S4<Var> o = mvec(CR, L[c]);
                        for (int k = 0; k < 4; ++k) {
                            double w = dI[((a * npix + ip) * 3 + c) * 4 + k] * inv_spp;
                            if (w != 0.0) J0 = J0 + o.s[k] * w;
                        }
                    }
                }
                g_tape_total += (double)g_tape.size();
                tape_backward(J0, 1.0, grad);
                g_tape.clear();
            } else {
                // ---- cached suffix replay
                // primal pass: E_v, W_v per vertex and the backward fold into suffixes L[v]
                std::vector<VEval<double>> ev(n);
                for (int v = 0; v < n; ++v) ev[v] = eval_vertex<double>(s, pd, path.vs[v]);
                std::vector<std::array<S4<double>, 3>> Lc(n + 1);
                for (int c = 0; c < 3; ++c) Lc[n][c] = szero<double>();
                for (int v = n - 1; v >= 0; --v)
                    for (int c = 0; c < 3; ++c) {
                        S4<double> wl = mvec(ev[v].W[c], Lc[v + 1][c]);
                        for (int k = 0; k < 4; ++k) Lc[v][c].s[k] = ev[v].E[c].s[k] + wl.s[k];
                    }
                // camera-filter term and the initial adjoint row a = sum_a dI_a^T C_a R / spp
                double arow[3][4] = {};
                for (int a = 0; a < A; ++a) {
                    g_tape.clear();
                    Var th = J.filter == FILTER_NONE ? Var(0.0) : pvar.at(lay.theta + a);
                    M4<Var> Cv = camera_filter<Var>(J.filter, th);
                    Var Jt(0.0);
                    for (int c = 0; c < 3; ++c) {
                        S4<double> raw = mvec(Rc, Lc[0][c]);
                        S4<Var> o = mvec(Cv, raw);
                        for (int k = 0; k < 4; ++k) {
                            double w = dI[((a * npix + ip) * 3 + c) * 4 + k] * inv_spp;
                            if (w == 0.0) continue;
                            Jt = Jt + o.s[k] * w;
                            for (int j = 0; j < 4; ++j) {
                                double crj = 0.0;
                                for (int q = 0; q < 4; ++q) crj += Cv.m[k][q].v * Rc.m[q][j];
                                arow[c][j] += w * crj;
                            }
                        }
                    }
                    tape_backward(Jt, 1.0, grad);
                    g_tape.clear();
                }
                // adjoint replay: local derivative at vertex v times the cached suffix L[v+1]
                for (int v = 0; v < n; ++v) {
                    g_tape.clear();
                    VEval<Var> e = eval_vertex<Var>(s, pvar, path.vs[v]);
                    Var Jv(0.0);
                    for (int c = 0; c < 3; ++c) {
                        S4<Var> wl = mvec(e.W[c], Lc[v + 1][c]);
                        for (int k = 0; k < 4; ++k) {
                            if (arow[c][k] == 0.0) continue;
                            Jv = Jv + (e.E[c].s[k] + wl.s[k]) * arow[c][k];
                        }
                    }
                    tape_backward(Jv, 1.0, grad);
                    g_tape.clear();
                    double na[3][4];
                    for (int c = 0; c < 3; ++c)
                        for (int j = 0; j < 4; ++j) {
                            double sacc = 0.0;
                            for (int k = 0; k < 4; ++k) sacc += arow[c][k] * ev[v].W[c].m[k][j];
                            na[c][j] = sacc;
                        }
                    std::memcpy(arow, na, sizeof(na));
                }
            }
        }
    }
    return 0;
}

}  // extern "C"

// Basic polarized PRB (P-PRB, Sec. 4.1 with the noise regularization of Sec. 4.2): the
// baseline the paper shows to fail for rank-deficient, polarization-aware operators, kept
// here to demonstrate that failure against the exact routes.  The replay knows only the
// path's total L[1] and recovers each suffix by removing the vertex,
//     L[v+1] = (W_v + u_v I)^-1 (L[v] - E_v),   u_v ~ N(0, sigma),
// u_v drawn per (path, vertex) from Philox (key seed ^ 0x5bd1e995, pass 3) by Box-Muller.
// flags bit 0: the noise also enters the primal fold and the adjoint's throughput (the
// paper's reading: the same u in both phases); clear, only the inversion is regularized.
// flags bit 1: the fold and the recovery run in single precision (the precision of a
// GPU renderer); the local derivative itself is taken in double either way.
template <typename T>
static bool solve4(T m[4][5], T x[4]) {
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r) if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
        if (m[piv][c] == T(0)) return false;
        if (piv != c) for (int j = 0; j < 5; ++j) std::swap(m[c][j], m[piv][j]);
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            T f = m[r][c] / m[c][c];
            for (int j = c; j < 5; ++j) m[r][j] -= f * m[c][j];
        }
    }
    for (int i = 0; i < 4; ++i) x[i] = m[i][4] / m[i][i];
    return true;
}

template <typename T>
static void pprb_path(const Scene& s, const Params<double>& pd, const Params<Var>& pvar, const Layout& lay,
                      const JobDesc& J, int A, int64_t ip, int64_t npix, int64_t pix, int smp, const double* dI,
                      double* grad, double sigma, bool primal_noise) {
    Path path = sample_path(s, pd, J, pix, smp);
    int n = (int)path.vs.size();
    M4<double> Rc = camera_rot(s, J.cam, path.d1);
    const double inv_spp = 1.0 / J.spp;
    uint64_t pid = (uint64_t)(pix * J.spp + smp);
    std::vector<VEval<double>> ev(n);
    std::vector<double> u(n);
    for (int v = 0; v < n; ++v) {
        ev[v] = eval_vertex<double>(s, pd, path.vs[v]);
        Uniforms un = draw(J.seed ^ 0x5bd1e995ULL, 3, J.stream, pid, (uint64_t)v);
        u[v] = sigma * std::sqrt(-2.0 * std::log(std::max(un.u[0], 1e-300))) * std::cos(2.0 * M_PI * un.u[1]);
    }
    const double up = primal_noise ? 1.0 : 0.0;
    // phase 1: the path's total, folded from the light end
    T L[3][4] = {};
    for (int v = n - 1; v >= 0; --v)
        for (int c = 0; c < 3; ++c) {
            T nx[4];
            for (int k = 0; k < 4; ++k) {
                T acc = (T)ev[v].E[c].s[k] + (T)(up * u[v]) * L[c][k];
                for (int j = 0; j < 4; ++j) acc += (T)ev[v].W[c].m[k][j] * L[c][j];
                nx[k] = acc;
            }
            for (int k = 0; k < 4; ++k) L[c][k] = nx[k];
        }
    // camera: the filter's own derivative and the adjoint row entering the first vertex
    double arow[3][4] = {};
    for (int a = 0; a < A; ++a) {
        g_tape.clear();
        Var th = J.filter == FILTER_NONE ? Var(0.0) : pvar.at(lay.theta + a);
        M4<Var> Cv = camera_filter<Var>(J.filter, th);
        Var Jt(0.0);
        for (int c = 0; c < 3; ++c) {
            S4<double> tot;
            for (int k = 0; k < 4; ++k) tot.s[k] = (double)L[c][k];
            S4<Var> o = mvec(Cv, mvec(Rc, tot));
            for (int k = 0; k < 4; ++k) {
                double w = dI[((a * npix + ip) * 3 + c) * 4 + k] * inv_spp;
                if (w == 0.0) continue;
                Jt = Jt + o.s[k] * w;
                for (int j = 0; j < 4; ++j) {
                    double crj = 0.0;
                    for (int q = 0; q < 4; ++q) crj += Cv.m[k][q].v * Rc.m[q][j];
                    arow[c][j] += w * crj;
                }
            }
        }
        tape_backward(Jt, 1.0, grad);
        g_tape.clear();
    }
    // phase 2: replay, recovering each suffix by inversion
    for (int v = 0; v < n; ++v) {
        S4<double> Ln[3];
        for (int c = 0; c < 3; ++c) {
            T m[4][5], x[4];
            for (int k = 0; k < 4; ++k) {
                for (int j = 0; j < 4; ++j) m[k][j] = (T)ev[v].W[c].m[k][j] + (k == j ? (T)u[v] : T(0));
                m[k][4] = L[c][k] - (T)ev[v].E[c].s[k];
            }
            if (!solve4(m, x)) for (int k = 0; k < 4; ++k) x[k] = T(0);
            for (int k = 0; k < 4; ++k) { L[c][k] = x[k]; Ln[c].s[k] = (double)x[k]; }
        }
        g_tape.clear();
        VEval<Var> e = eval_vertex<Var>(s, pvar, path.vs[v]);
        Var Jv(0.0);
        for (int c = 0; c < 3; ++c) {
            S4<Var> wl = mvec(e.W[c], Ln[c]);
            for (int k = 0; k < 4; ++k)
                if (arow[c][k] != 0.0) Jv = Jv + (e.E[c].s[k] + wl.s[k]) * arow[c][k];
        }
        tape_backward(Jv, 1.0, grad);
        g_tape.clear();
        double na[3][4];
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 4; ++j) {
                double acc = arow[c][j] * up * u[v];
                for (int k = 0; k < 4; ++k) acc += arow[c][k] * ev[v].W[c].m[k][j];
                na[c][j] = acc;
            }
        std::memcpy(arow, na, sizeof(na));
    }
}

extern "C" {
int orc_gradient_pprb(void* sc, const int64_t* job, const int64_t* pixels, int64_t npix, const double* Pd,
                      const int64_t* layout, const double* dI, double* grad, double sigma, int flags) {
    const Scene& s = *(const Scene*)sc;
    JobDesc J = job_from(job);
    Layout lay = layout_from(layout);
    Params<double> pd{Pd, lay};
    Params<Var> pvar{Pd, lay};
    int A = J.filter == FILTER_NONE ? 1 : J.nang;
    bool primal_noise = flags & 1, single = flags & 2;
    for (int64_t ip = 0; ip < npix; ++ip)
        for (int smp = 0; smp < J.spp; ++smp) {
            if (single) pprb_path<float>(s, pd, pvar, lay, J, A, ip, npix, pixels[ip], smp, dI, grad, sigma, primal_noise);
            else pprb_path<double>(s, pd, pvar, lay, J, A, ip, npix, pixels[ip], smp, dI, grad, sigma, primal_noise);
        }
    return 0;
}

// Hybrid cached replay (Sec. 4.4, Eq. hybrid_decision).  The primal pass keeps the suffix
// L[c] only at checkpoints c = 0, k, 2k, ... (L[n] = 0).  The replay of a block starting at
// checkpoint c carries the detached block throughput bt = W_c ... W_v and the block's
// emitted part eb = sum_{j=c..v} W_c ... W_{j-1} E_j, so that L[c] = eb + bt L[v+1].  A
// suffix L[v+1] that is not a checkpoint is recovered per colour channel, in this order:
//   DI(bt) < gamma            : scalar PRB, s0 = (L[c] - eb)_0 / bt_00, polarization dropped;
//   |det bt| > eps            : bt^-1 (L[c] - eb);
//   otherwise                 : recomputation -- the vertices v+1 .. (next checkpoint - 1)
//                               are evaluated again and folded onto the next checkpoint.
// DI is the depolarization index of Gil and Bernabeu, sqrt(sum m_ij^2 - m_00^2) /
// (sqrt(3) m_00): 0 for an ideal depolarizer, 1 for a non-depolarizing operator.
// routes[0..3] += channel-vertices served from a checkpoint, by scalar PRB, by inversion,
// by recomputation.
static double depol_index(const M4<double>& m) {
    if (!(m.m[0][0] > 0.0)) return HUGE_VAL;
    double s2 = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) s2 += m.m[i][j] * m.m[i][j];
    return std::sqrt(std::max(0.0, s2 - m.m[0][0] * m.m[0][0])) / (std::sqrt(3.0) * m.m[0][0]);
}
static double det4(const M4<double>& A) {
    double m[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) m[i][j] = A.m[i][j];
    double d = 1.0;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r) if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0) return 0.0;
        if (piv != c) { for (int j = 0; j < 4; ++j) std::swap(m[c][j], m[piv][j]); d = -d; }
        d *= m[c][c];
        for (int r = c + 1; r < 4; ++r) {
            double f = m[r][c] / m[c][c];
            for (int j = c; j < 4; ++j) m[r][j] -= f * m[c][j];
        }
    }
    return d;
}

extern "C" int orc_gradient_hybrid(void* sc, const int64_t* job, const int64_t* pixels, int64_t npix,
                                   const double* Pd, const int64_t* layout, const double* dI, double* grad,
                                   int k, double gamma, double eps, double* routes) {
    const Scene& s = *(const Scene*)sc;
    if (k < 1) return -1;
    JobDesc J = job_from(job);
    Layout lay = layout_from(layout);
    Params<double> pd{Pd, lay};
    Params<Var> pvar{Pd, lay};
    int A = J.filter == FILTER_NONE ? 1 : J.nang;
    for (int64_t ip = 0; ip < npix; ++ip) {
        int64_t pix = pixels[ip];
        for (int smp = 0; smp < J.spp; ++smp) {
            Path path = sample_path(s, pd, J, pix, smp);
            int n = (int)path.vs.size();
            M4<double> Rc = camera_rot(s, J.cam, path.d1);
            const double inv_spp = 1.0 / J.spp;
            // primal pass: fold, keeping the suffix only at the checkpoints
            int nck = n / k + 2;
            std::vector<std::array<S4<double>, 3>> Lck(nck);
            for (auto& a : Lck) for (int c = 0; c < 3; ++c) a[c] = szero<double>();
            {
                S4<double> L[3] = {szero<double>(), szero<double>(), szero<double>()};
                for (int v = n - 1; v >= 0; --v) {
                    VEval<double> e = eval_vertex<double>(s, pd, path.vs[v]);
                    for (int c = 0; c < 3; ++c) {
                        S4<double> wl = mvec(e.W[c], L[c]);
                        for (int q = 0; q < 4; ++q) L[c].s[q] = e.E[c].s[q] + wl.s[q];
                    }
                    if (v % k == 0) for (int c = 0; c < 3; ++c) Lck[v / k][c] = L[c];
                }
            }
            auto suffix_at_ck = [&](int idx, int c) -> S4<double> {   // L[idx], idx a checkpoint or n
                return idx >= n ? szero<double>() : Lck[idx / k][c];
            };
            // camera-filter term and the initial adjoint row
            double arow[3][4] = {};
            for (int a = 0; a < A; ++a) {
                g_tape.clear();
                Var th = J.filter == FILTER_NONE ? Var(0.0) : pvar.at(lay.theta + a);
                M4<Var> Cv = camera_filter<Var>(J.filter, th);
                Var Jt(0.0);
                for (int c = 0; c < 3; ++c) {
                    S4<Var> o = mvec(Cv, mvec(Rc, suffix_at_ck(0, c)));
                    for (int q = 0; q < 4; ++q) {
                        double w = dI[((a * npix + ip) * 3 + c) * 4 + q] * inv_spp;
                        if (w == 0.0) continue;
                        Jt = Jt + o.s[q] * w;
                        for (int j = 0; j < 4; ++j) {
                            double crj = 0.0;
                            for (int r = 0; r < 4; ++r) crj += Cv.m[q][r].v * Rc.m[r][j];
                            arow[c][j] += w * crj;
                        }
                    }
                }
                tape_backward(Jt, 1.0, grad);
                g_tape.clear();
            }
            // replay
            M4<double> bt[3];
            S4<double> eb[3], Lblk[3];
            for (int v = 0; v < n; ++v) {
                if (v % k == 0)
                    for (int c = 0; c < 3; ++c) { bt[c] = M4<double>::ident(); eb[c] = szero<double>(); Lblk[c] = suffix_at_ck(v, c); }
                VEval<double> ev = eval_vertex<double>(s, pd, path.vs[v]);
                for (int c = 0; c < 3; ++c) {
                    S4<double> be = mvec(bt[c], ev.E[c]);
                    for (int q = 0; q < 4; ++q) eb[c].s[q] += be.s[q];
                    bt[c] = mmul(bt[c], ev.W[c]);
                }
                S4<double> Ln[3];
                const int next = (v / k + 1) * k;
                for (int c = 0; c < 3; ++c) {
                    if (v + 1 == next || v + 1 >= n) { Ln[c] = suffix_at_ck(v + 1, c); routes[0] += 1; continue; }
                    S4<double> r;
                    for (int q = 0; q < 4; ++q) r.s[q] = Lblk[c].s[q] - eb[c].s[q];
                    double di = depol_index(bt[c]);
                    if (di < gamma) {
                        Ln[c] = szero<double>();
                        Ln[c].s[0] = r.s[0] / bt[c].m[0][0];
                        routes[1] += 1;
                    } else if (std::fabs(det4(bt[c])) > eps) {
                        double m[4][5], x[4];
                        for (int i = 0; i < 4; ++i) { for (int j = 0; j < 4; ++j) m[i][j] = bt[c].m[i][j]; m[i][4] = r.s[i]; }
                        solve4(m, x);
                        for (int q = 0; q < 4; ++q) Ln[c].s[q] = x[q];
                        routes[2] += 1;
                    } else {
                        // trace on to the next checkpoint and fold onto its cached suffix
                        S4<double> acc = szero<double>();
                        M4<double> T = M4<double>::ident();
                        for (int j = v + 1; j < std::min(next, n); ++j) {
                            VEval<double> ej = eval_vertex<double>(s, pd, path.vs[j]);
                            S4<double> te = mvec(T, ej.E[c]);
                            for (int q = 0; q < 4; ++q) acc.s[q] += te.s[q];
                            T = mmul(T, ej.W[c]);
                        }
                        S4<double> tl = mvec(T, suffix_at_ck(next, c));
                        for (int q = 0; q < 4; ++q) Ln[c].s[q] = acc.s[q] + tl.s[q];
                        routes[3] += 1;
                    }
                }
                g_tape.clear();
                VEval<Var> e = eval_vertex<Var>(s, pvar, path.vs[v]);
                Var Jv(0.0);
                for (int c = 0; c < 3; ++c) {
                    S4<Var> wl = mvec(e.W[c], Ln[c]);
                    for (int q = 0; q < 4; ++q)
                        if (arow[c][q] != 0.0) Jv = Jv + (e.E[c].s[q] + wl.s[q]) * arow[c][q];
                }
                tape_backward(Jv, 1.0, grad);
                g_tape.clear();
                double na[3][4];
                for (int c = 0; c < 3; ++c)
                    for (int j = 0; j < 4; ++j) {
                        double acc = 0.0;
                        for (int q = 0; q < 4; ++q) acc += arow[c][q] * ev.W[c].m[q][j];
                        na[c][j] = acc;
                    }
                std::memcpy(arow, na, sizeof(na));
            }
        }
    }
    return 0;
}

// ---------------------------------------------------------------- unit probes
void orc_philox(const uint64_t* ctr, const uint64_t* key, uint64_t* out) { philox4x64_10(ctr, key, out); }
void orc_uniforms(uint64_t seed, uint64_t pass, uint64_t stream, uint64_t path, uint64_t vertex, double* u) {
    Uniforms r = draw(seed, pass, stream, path, vertex);
    for (int k = 0; k < 8; ++k) u[k] = r.u[k];
}
// Fresnel reflection (A,B,C,S) for eta_i real, eta_t complex
void orc_fresnel_reflect(double cos_i, double eta_i, double eta_t_re, double eta_t_im, double* abcs) {
    FresnelABCS<double> f = fresnel_reflect<double>(cos_i, eta_i, Cx<double>{eta_t_re, eta_t_im});
    abcs[0] = f.A; abcs[1] = f.B; abcs[2] = f.C; abcs[3] = f.S;
}
void orc_fresnel_transmit(double cos_i, double eta_i, double eta_t, double* abcs) {
    FresnelABCS<double> f = fresnel_transmit<double>(cos_i, eta_i, eta_t);
    abcs[0] = f.A; abcs[1] = f.B; abcs[2] = f.C; abcs[3] = f.S;
}
void orc_camera_filter(int filter, double theta, double* m16) {
    M4<double> C = camera_filter<double>(filter, theta);
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) m16[4 * i + j] = C.m[i][j];
}
// GGX normal distribution D(cos_h) and Smith masking G1(cos_v, cos_vh) (Walter et al. 2007)
void orc_ggx(double cos_h, double cos_v, double cos_vh, double alpha, double* out) {
    out[0] = ggx_D<double>(cos_h, alpha);
    out[1] = ggx_G1<double>(cos_v, cos_vh, alpha);
}
// depolarization index (Gil and Bernabeu) of a Mueller matrix m16, row-major
double orc_depol_index(const double* m16) {
    M4<double> m;
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) m.m[i][j] = m16[4 * i + j];
    return depol_index(m);
}
// bilinear texture lookup of channel c at (u, v) in a w x h texture of ch channels, texels
// [h][w][ch] in `texels`
double orc_tex_lookup(int w, int h, int ch, const double* texels, int c, double u, double v) {
    Scene s;
    s.tex.push_back({0, w, h, ch});
    Layout lay{};
    Params<double> P{texels, lay};
    return tex_lookup<double>(s, P, 0, c, u, v);
}
void orc_csqrt(double re, double im, double* out) {
    Cx<double> r = csqrt(Cx<double>{re, im});
    out[0] = r.re; out[1] = r.im;
}
// closest hit: returns prim (-1 miss), t, and, with brute != 0, ignores the BVH
int orc_closest(void* sc, const double* o, const double* d, int brute, double* t_out) {
    const Scene& s = *(const Scene*)sc;
    Ray r{ld3(o), ld3(d)};
    Hit h;
    if (brute) {
        h.t = 1e300; h.prim = -1;
        for (int f = 0; f < s.F(); ++f) {
            double b1, b2, t = tri_hit(s, f, r, b1, b2);
            if (t > 0.0 && (t < h.t || (t == h.t && f < h.prim))) { h.t = t; h.prim = f; }
        }
        for (int k = 0; k < (int)s.smat.size(); ++k) {
            double t = sph_hit(s, k, r, 1e300);
            if (t > 0.0 && t < h.t) { h.t = t; h.prim = s.F() + k; }
        }
    } else closest(s, r, h);
    *t_out = h.t;
    return h.prim;
}
void orc_stats(double* out, int reset) {
    out[0] = g_stats.rays; out[1] = g_stats.shadow_rays; out[2] = g_stats.vertices; out[3] = g_stats.nodes;
    out[4] = g_stats.tri_tests; out[5] = g_stats.sph_tests; out[6] = g_stats.paths; out[7] = (double)g_tape_peak;
    out[8] = g_tape_total;
    if (reset) { g_stats = Stats{}; g_tape_peak = 0; g_tape_total = 0; }
}

}  // extern "C"
