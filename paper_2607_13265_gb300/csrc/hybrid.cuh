// Hybrid cached replay (Sec. 4.4, Eq. hybrid_decision): the adjoint megakernel that keeps
// the suffix L[c] only at checkpoints c = 0, K, 2K, ... instead of at every vertex.
//
// Per path, one thread:
//   pass 0 (detached): for every block of K vertices starting at checkpoint c it forms the
//     block's emitted part e_b = sum_j W_c..W_{j-1} E_j and throughput T_b = W_c..W_{c+K-1}
//     (full 4x4 per colour channel) and, at every vertex v inside the block, decides how the
//     replay will recover L[v+1] from the running throughput bt = W_c..W_v:
//       DI(bt) < gamma  -> scalar PRB (s0 only);  |det bt| > eps -> bt^-1 (L[c] - eb);
//       otherwise       -> recomputation;
//     a backward fold over the blocks, L[c_b] = e_b + T_b L[c_{b+1}], leaves the checkpoints.
//   pass 1 (replay with dual numbers): vertex v takes L[v+1] from a checkpoint when v+1 is
//     one, else by the route chosen in pass 0; a block with a recomputed vertex is first
//     traced again (detached) from the saved walk state up to the next checkpoint, its
//     E/W folded onto that checkpoint's suffix.
// Per-thread memory: (MAXD/K + 2) x 60 floats of block data, K x 31 floats of look-ahead,
// MAXD route bytes -- instead of the MAXD x 31 floats of the fully cached replay.  The
// visitor works on whatever memory its pointers give it: the megakernel's thread-local
// arrays, or a path's records in the wavefront's workspace (wf_hybrid.cu).
#pragma once

#include "trace.cuh"

namespace dppt {

// M <- M W_c for a row-major 4x4 M (each row r: r^T W_c)
__device__ __forceinline__ void m4_times_compact(float* M, const Compact<float>& W, int c) {
#pragma unroll
    for (int r = 0; r < 4; ++r) compact_row(W, c, M + 4 * r);
}

// depolarization index of Gil and Bernabeu: sqrt(sum m_ij^2 - m_00^2) / (sqrt(3) m_00)
__device__ __forceinline__ float depol_index(const float* M) {
    if (!(M[0] > 0.0f)) return INFINITY;
    float s2 = 0.0f;
#pragma unroll
    for (int k = 1; k < 16; ++k) s2 = fmaf(M[k], M[k], s2);
    return sqrtf(s2) / (1.7320508f * M[0]);
}

// Gaussian elimination with partial pivoting on [M | b] (b may be null): returns det M and,
// when b is given and M is not singular, overwrites b with M^-1 b.
static __device__ __noinline__ float m4_eliminate(const float* M, float* b) {
    float m[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int q = 0; q < 4; ++q) m[r][q] = M[4 * r + q];
        m[r][4] = b ? b[r] : 0.0f;
    }
    float det = 1.0f;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabsf(m[r][c]) > fabsf(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0f) return 0.0f;
        if (piv != c) {
            for (int q = 0; q < 5; ++q) { float t = m[c][q]; m[c][q] = m[piv][q]; m[piv][q] = t; }
            det = -det;
        }
        det *= m[c][c];
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            float f = m[r][c] / m[c][c];
            for (int q = c; q < 5; ++q) m[r][q] = fmaf(-f, m[c][q], m[r][q]);
        }
    }
    if (b)
        for (int r = 0; r < 4; ++r) b[r] = m[r][4] / m[r][r];
    return det;
}

enum : unsigned { kRouteNone = 0, kRouteScalar = 1, kRouteInverse = 2, kRouteRecompute = 3 };

template <int MAXD, int K>
struct HybVis {
    static constexpr int NB = MAXD / K + 2;
    const DScene* S;
    const DParams* P;
    const DGrads* G;
    float* sgrad;
    float (*ck)[60];        // per block: pass 0 e_b (0..11) | T_b (12..59); after the fold L[c_b] (0..11)
    unsigned char* route;   // per vertex: 2 bits per channel
    float (*blk)[31];       // look-ahead of the current block: E|W per slot, folded into suffixes
    float* bt;              // [48] replay: throughput since the block's checkpoint
    float* ebr;             // [12] replay: emission since the block's checkpoint
    unsigned* flags;        // blocks holding a recomputed vertex
    float a[3][4];
    float gamma, eps;
    int n, i, phase, la, blk_base;
    int cap;                // vertices cached at most (MAXD in the megakernel, the wave's depth in the wavefront)

    __device__ __forceinline__ bool flagged(int b) const { return (flags[b >> 5] >> (b & 31)) & 1u; }

    __device__ __forceinline__ void operator()(const VCtx& vc) {
        if (phase == 0) { cache_vertex(vc); return; }
        if (phase == 2) { look_ahead(vc); return; }
        if (i >= n) return;
        replay_vertex(vc);
        ++i;
    }

    __device__ void cache_vertex(const VCtx& vc) {
        if (n >= cap) return;
        float E[3][4];
        Compact<float> W;
        eval_vertex<float>(*S, *P, vc, E, W, nullptr);
        const int v = n, b = v / K;
        float* cb = ck[b];
        if (v % K == 0) {
            for (int k = 0; k < 60; ++k) cb[k] = 0.0f;
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < 4; ++r) cb[12 + 16 * c + 5 * r] = 1.0f;
        }
        for (int c = 0; c < 3; ++c) {
            const float* T = cb + 12 + 16 * c;
            for (int r = 0; r < 4; ++r)
                cb[4 * c + r] += T[4 * r] * E[c][0] + T[4 * r + 1] * E[c][1] + T[4 * r + 2] * E[c][2] +
                                 T[4 * r + 3] * E[c][3];
        }
        unsigned rb = 0u;
        if (vc.scatter) {
            for (int c = 0; c < 3; ++c) m4_times_compact(cb + 12 + 16 * c, W, c);
            if ((v + 1) % K != 0) {
                for (int c = 0; c < 3; ++c) {
                    const float* T = cb + 12 + 16 * c;
                    unsigned r;
                    if (depol_index(T) < gamma) r = kRouteScalar;
                    else if (fabsf(m4_eliminate(T, nullptr)) > eps) r = kRouteInverse;
                    else r = kRouteRecompute;
                    rb |= r << (2 * c);
                    if (r == kRouteRecompute) flags[b >> 5] |= 1u << (b & 31);
                }
            }
        }
        route[v] = (unsigned char)rb;
        ++n;
    }

    // backward fold over the blocks; returns L[0] (the path's total) in L0
    __device__ void fold(float L0[12]) {
        float L[12];
        for (int k = 0; k < 12; ++k) L[k] = 0.0f;
        for (int b = (n + K - 1) / K - 1; b >= 0; --b) {
            float* cb = ck[b];
            float y[12];
            for (int c = 0; c < 3; ++c) {
                const float* T = cb + 12 + 16 * c;
                for (int r = 0; r < 4; ++r)
                    y[4 * c + r] = cb[4 * c + r] + T[4 * r] * L[4 * c] + T[4 * r + 1] * L[4 * c + 1] +
                                   T[4 * r + 2] * L[4 * c + 2] + T[4 * r + 3] * L[4 * c + 3];
            }
            for (int k = 0; k < 12; ++k) { L[k] = y[k]; cb[k] = y[k]; }
        }
        for (int k = 0; k < 12; ++k) L0[k] = L[k];
    }

    __device__ void look_ahead(const VCtx& vc) {
        const int s = la++;
        if (s < 1 || s >= K) return;
        float E[3][4];
        Compact<float> W;
        eval_vertex<float>(*S, *P, vc, E, W, nullptr);
        float* q = blk[s];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) q[4 * c + k] = E[c][k];
        q[12] = W.ri.c; q[13] = W.ri.s; q[14] = W.ro.c; q[15] = W.ro.s;
        for (int c = 0; c < 3; ++c) {
            q[16 + c] = W.A[c]; q[19 + c] = W.B[c]; q[22 + c] = W.C[c]; q[25 + c] = W.S[c]; q[28 + c] = W.D[c];
        }
    }

    // folds the look-ahead onto the next checkpoint: slot s then holds L[blk_base + s]
    __device__ void fold_block() {
        const int c0 = blk_base, top = min(c0 + K, n);
        float L[12];
        const bool has_next = c0 + K < n;
        for (int k = 0; k < 12; ++k) L[k] = has_next ? ck[(c0 + K) / K][k] : 0.0f;
        for (int j = top - 1; j >= c0 + 1; --j) {
            float* q = blk[j - c0];
            Compact<float> W;
            W.ri = {q[12], q[13]}; W.ro = {q[14], q[15]};
            for (int c = 0; c < 3; ++c) {
                W.A[c] = q[16 + c]; W.B[c] = q[19 + c]; W.C[c] = q[22 + c]; W.S[c] = q[25 + c]; W.D[c] = q[28 + c];
            }
            for (int c = 0; c < 3; ++c) {
                float y[4];
                compact_apply(W, c, &L[4 * c], y);
                for (int k = 0; k < 4; ++k) L[4 * c + k] = q[4 * c + k] + y[k];
            }
            for (int k = 0; k < 12; ++k) q[k] = L[k];
        }
    }

    __device__ void replay_vertex(const VCtx& vc) {
        float E[3][4];
        Compact<D3> W, f;
        eval_vertex<D3>(*S, *P, vc, E, W, &f);
        const int b = i / K, s = i % K;
        float Ln[3][4];
        if (i + 1 >= n) {
            for (int k = 0; k < 12; ++k) Ln[k >> 2][k & 3] = 0.0f;
        } else if ((i + 1) % K == 0) {
            for (int k = 0; k < 12; ++k) Ln[k >> 2][k & 3] = ck[(i + 1) / K][k];
        } else {
            // block throughput and emission so far (detached values)
            if (s == 0) {
                for (int k = 0; k < 48; ++k) bt[k] = (k & 15) % 5 == 0 ? 1.0f : 0.0f;
                for (int k = 0; k < 12; ++k) ebr[k] = 0.0f;
            }
            const Compact<float> Wv = compact_value(W);
            for (int c = 0; c < 3; ++c) {
                float* T = bt + 16 * c;
                for (int r = 0; r < 4; ++r)
                    ebr[4 * c + r] += T[4 * r] * E[c][0] + T[4 * r + 1] * E[c][1] + T[4 * r + 2] * E[c][2] +
                                      T[4 * r + 3] * E[c][3];
                m4_times_compact(T, Wv, c);
            }
            const unsigned rb = route[i];
            for (int c = 0; c < 3; ++c) {
                const unsigned r = (rb >> (2 * c)) & 3u;
                float x[4];
                for (int k = 0; k < 4; ++k) x[k] = ck[b][4 * c + k] - ebr[4 * c + k];
                if (r == kRouteScalar) {
                    Ln[c][0] = x[0] / bt[16 * c];
                    Ln[c][1] = Ln[c][2] = Ln[c][3] = 0.0f;
                } else if (r == kRouteInverse) {
                    m4_eliminate(bt + 16 * c, x);
                    for (int k = 0; k < 4; ++k) Ln[c][k] = x[k];
                } else if (r == kRouteRecompute) {
                    for (int k = 0; k < 4; ++k) Ln[c][k] = blk[s + 1][4 * c + k];
                } else {
                    for (int k = 0; k < 4; ++k) Ln[c][k] = 0.0f;
                }
            }
        }
        replay_vjp(*S, *P, *G, sgrad, vc, W, f, Ln, a);
    }
};

template <int MAXD, int K>
__global__ void __launch_bounds__(256, DPPT_MIN_BLOCKS_ADJOINT)
k_hybrid(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T,
         unsigned long long* counter, unsigned* status, int persistent, HybridCfg hc) {
    extern __shared__ float sgrad[];
    __shared__ long long s_chunk;
    sgrad_zero(S, sgrad);
    constexpr int NB = HybVis<MAXD, K>::NB;
    float ck[NB][60];
    unsigned char route[MAXD];
    float blk[K][31];
    float bt[48], ebr[12];
    unsigned flags[(NB + 31) / 32];
    WorkCount wc = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
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
        for (int k = 0; k < 12; ++k) raw[k] = 0.0f;
        if (active) {
            const long long pix = p / J.spp;
            HybVis<MAXD, K> vis;
            vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad;
            vis.ck = ck; vis.route = route; vis.blk = blk; vis.bt = bt; vis.ebr = ebr; vis.flags = flags;
            vis.gamma = hc.gamma; vis.eps = hc.eps;
            vis.n = 0; vis.i = 0; vis.la = 0; vis.blk_base = 0; vis.cap = MAXD;
            for (int k = 0; k < (NB + 31) / 32; ++k) flags[k] = 0u;
            Walk w;
            vis.phase = 0;
            walk_begin(S, J, (unsigned long long)p, pix, w);
            while (walk_step<HybVis<MAXD, K>, false>(S, P, J, (unsigned long long)p, w, vis, status, &wc)) {
            }
            float L0[12];
            vis.fold(L0);
            Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
            const float inv = 1.0f / (float)J.spp;
            for (int c = 0; c < 3; ++c) {
                float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
                rot_apply(Rc, v);
                for (int k = 0; k < 4; ++k) raw[4 * c + k] = v[k] * inv;
            }
            if (vis.n > 0) {
                const float* ds = J.dS + pix * 12;
                for (int c = 0; c < 3; ++c) {
                    float av[4] = {__ldg(ds + 4 * c) * inv, __ldg(ds + 4 * c + 1) * inv, __ldg(ds + 4 * c + 2) * inv,
                                   __ldg(ds + 4 * c + 3) * inv};
                    rot_apply_row(Rc, av);
                    for (int k = 0; k < 4; ++k) vis.a[c][k] = av[k];
                }
                vis.phase = 1;
                walk_begin(S, J, (unsigned long long)p, pix, w);
                for (;;) {
                    if (vis.i < vis.n && vis.i % K == 0 && vis.flagged(vis.i / K)) {
                        // trace the block again, detached, up to the next checkpoint
                        Walk w2 = w;
                        vis.phase = 2; vis.la = 0; vis.blk_base = vis.i;
                        while (vis.la < K &&
                               walk_step<HybVis<MAXD, K>, false>(S, P, J, (unsigned long long)p, w2, vis, status, &wc)) {
                        }
                        vis.fold_block();
                        vis.phase = 1;
                    }
                    if (!walk_step<HybVis<MAXD, K>, false>(S, P, J, (unsigned long long)p, w, vis, status, &wc)) break;
                }
            }
            if (J.sig) J.sig[p] = fnv(w.sig, (unsigned)w.nv);
        }
        if (J.raw) {
            __syncwarp();
            pixel_reduce(J, J.raw, p, active, raw);
        }
        if (!persistent) break;
    }
    sgrad_flush(S, G, sgrad);
}

template <int MAXD, int K>
cudaError_t launch_hybrid_t(const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,
                            const LaunchCfg& L, unsigned long long* counter, unsigned* status, HybridCfg hc,
                            cudaStream_t st) {
    const int pers = L.schedule == DPPT_SCHED_PERSISTENT;
    long long g = pers ? L.grid : T.total_chunks;
    if (g <= 0) return cudaSuccess;
    if (g > 0x7fffffffLL) g = 0x7fffffffLL;
    const size_t sm = sgrad_bytes(S);
    k_hybrid<MAXD, K><<<(int)g, L.block, sm, st>>>(S, P, G, T, counter, status, pers, hc);
    return cudaGetLastError();
}

// one translation unit per checkpoint interval instantiates the kernels of every depth bucket
#define DPPT_HYBRID_INTERVAL(K)                                                                                     \
    cudaError_t launch_hybrid_##K(int bucket, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, \
                                  const LaunchCfg& L, unsigned long long* counter, unsigned* status, HybridCfg hc, \
                                  cudaStream_t st) {                                                              \
        switch (bucket) {                                                                                         \
            case 8: return launch_hybrid_t<8, K>(S, P, G, T, L, counter, status, hc, st);                         \
            case 16: return launch_hybrid_t<16, K>(S, P, G, T, L, counter, status, hc, st);                       \
            case 32: return launch_hybrid_t<32, K>(S, P, G, T, L, counter, status, hc, st);                       \
            case 64: return launch_hybrid_t<64, K>(S, P, G, T, L, counter, status, hc, st);                       \
            case 128: return launch_hybrid_t<128, K>(S, P, G, T, L, counter, status, hc, st);                     \
        }                                                                                                         \
        return cudaErrorInvalidValue;                                                                             \
    }                                                                                                             \
    static const void* hybrid_fn_##K(int bucket) {                                                                \
        switch (bucket) {                                                                                         \
            case 8: return reinterpret_cast<const void*>(&k_hybrid<8, K>);                                        \
            case 16: return reinterpret_cast<const void*>(&k_hybrid<16, K>);                                      \
            case 32: return reinterpret_cast<const void*>(&k_hybrid<32, K>);                                      \
            case 64: return reinterpret_cast<const void*>(&k_hybrid<64, K>);                                      \
            case 128: return reinterpret_cast<const void*>(&k_hybrid<128, K>);                                    \
        }                                                                                                         \
        return nullptr;                                                                                           \
    }                                                                                                             \
    cudaError_t hybrid_attributes_##K(int bucket, cudaFuncAttributes* a) {                                        \
        const void* f = hybrid_fn_##K(bucket);                                                                    \
        return f ? cudaFuncGetAttributes(a, f) : cudaErrorInvalidValue;                                          \
    }                                                                                                             \
    int hybrid_occupancy_##K(int bucket, int block, size_t smem) {                                                \
        int nb = 0;                                                                                               \
        const void* f = hybrid_fn_##K(bucket);                                                                    \
        if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem) != cudaSuccess) return 0;     \
        return nb;                                                                                                \
    }

}  // namespace dppt
