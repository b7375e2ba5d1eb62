// Basic polarized PRB (Sec. 4.1 with the noise regularization of Sec. 4.2): the baseline
// the paper compares against, as a cache-free adjoint megakernel (one thread per path).
//
//   pass 0: the path's total, accumulated forward with the noised throughput
//           beta <- beta (W_v + u_v I) (full 4x4 per colour channel): L = sum_v beta_v E_v;
//   pass 1: the replay recovers each suffix by removing the vertex,
//           L[v+1] = (W_v + u_v I)^-1 (L[v] - E_v), differentiates the vertex with dual
//           numbers against it and advances the adjoint row a <- a (W_v + u_v I).
// u_v ~ N(0, sigma) per (path, vertex): Philox with key (seed ^ 0x5bd1e995) ^ (3 * golden
// ratio constant) and the job's stream, counter (path, vertex, 0, 0), Box-Muller on the
// first two uniforms.  The same noise enters both passes.  Memory per thread: the 48-float
// throughput of pass 0, independent of the path depth.  Exact only where the factors are
// invertible (Sec. 4.1): it is the failure baseline, not a product path.
#include "hybrid.cuh"

namespace dppt {

struct PprbVis {
    const DScene* S;
    const DParams* P;
    const DGrads* G;
    float* sgrad;
    float* beta;          // [48] pass 0: noised throughput
    float L[12];          // pass 0: the running total; pass 1: the suffix L[v]
    float a[3][4];
    float sigma;
    unsigned long long kn, k1, pid;
    int n, i, phase;

    __device__ __forceinline__ float noise(int v) const {
        const U8 u = draw8(kn, k1, pid, (unsigned)v);
        return sigma * sqrtf(-2.0f * logf(fmaxf(u.u[0], 1e-30f))) * cosf(2.0f * kPi * u.u[1]);
    }

    __device__ __forceinline__ void operator()(const VCtx& vc) {
        if (phase == 0) { total_vertex(vc); return; }
        if (i >= n) return;
        replay_vertex(vc);
        ++i;
    }

    __device__ void total_vertex(const VCtx& vc) {
        float E[3][4];
        Compact<float> W;
        eval_vertex<float>(*S, *P, vc, E, W, nullptr);
        const float u = noise(n);
        for (int c = 0; c < 3; ++c) {
            float* B = beta + 16 * c;
            for (int r = 0; r < 4; ++r)
                L[4 * c + r] += B[4 * r] * E[c][0] + B[4 * r + 1] * E[c][1] + B[4 * r + 2] * E[c][2] + B[4 * r + 3] * E[c][3];
            if (vc.scatter) {
                float old[16];
                for (int k = 0; k < 16; ++k) old[k] = B[k];
                m4_times_compact(B, W, c);
                for (int k = 0; k < 16; ++k) B[k] = fmaf(u, old[k], B[k]);
            }
        }
        ++n;
    }

    __device__ void replay_vertex(const VCtx& vc) {
        float E[3][4];
        Compact<D3> W, f;
        eval_vertex<D3>(*S, *P, vc, E, W, &f);
        const Compact<float> Wv = compact_value(W);
        const float u = noise(i);
        float Ln[3][4];
        for (int c = 0; c < 3; ++c) {
            // (W_v + u I) column by column, then the inversion
            float M[16];
            for (int j = 0; j < 4; ++j) {
                float e[4] = {0.0f, 0.0f, 0.0f, 0.0f}, y[4];
                e[j] = 1.0f;
                compact_apply(Wv, c, e, y);
                for (int r = 0; r < 4; ++r) M[4 * r + j] = y[r] + (r == j ? u : 0.0f);
            }
            float x[4];
            for (int k = 0; k < 4; ++k) x[k] = L[4 * c + k] - E[c][k];
            if (m4_eliminate(M, x) == 0.0f)
                for (int k = 0; k < 4; ++k) x[k] = 0.0f;
            for (int k = 0; k < 4; ++k) Ln[c][k] = x[k];
        }
        float a_old[3][4];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) a_old[c][k] = a[c][k];
        replay_vjp(*S, *P, *G, sgrad, vc, W, f, Ln, a);     // a <- a W_v
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) {
                a[c][k] = fmaf(u, a_old[c][k], a[c][k]);
                L[4 * c + k] = Ln[c][k];
            }
    }
};

__global__ void __launch_bounds__(256, DPPT_MIN_BLOCKS_ADJOINT)
k_pprb(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T,
       unsigned long long* counter, unsigned* status, int persistent, float sigma) {
    extern __shared__ float sgrad[];
    __shared__ long long s_chunk;
    sgrad_zero(S, sgrad);
    float beta[48];
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
            PprbVis vis;
            vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad; vis.beta = beta;
            vis.sigma = sigma; vis.kn = J.kn; vis.k1 = J.k1; vis.pid = (unsigned long long)p;
            vis.n = 0; vis.i = 0;
            for (int k = 0; k < 12; ++k) vis.L[k] = 0.0f;
            for (int k = 0; k < 48; ++k) beta[k] = (k & 15) % 5 == 0 ? 1.0f : 0.0f;
            Walk w;
            vis.phase = 0;
            walk_begin(S, J, (unsigned long long)p, pix, w);
            while (walk_step<PprbVis, false>(S, P, J, (unsigned long long)p, w, vis, status, &wc)) {
            }
            Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
            const float inv = 1.0f / (float)J.spp;
            for (int c = 0; c < 3; ++c) {
                float v[4] = {vis.L[4 * c], vis.L[4 * c + 1], vis.L[4 * c + 2], vis.L[4 * c + 3]};
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
                while (walk_step<PprbVis, false>(S, P, J, (unsigned long long)p, w, vis, status, &wc)) {
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

cudaError_t launch_pprb(const DScene& S, const DParams& P, const DGrads& G, const JobTable& T, const LaunchCfg& L,
                        unsigned long long* counter, unsigned* status, float sigma, cudaStream_t st) {
    const int pers = L.schedule == DPPT_SCHED_PERSISTENT;
    long long g = pers ? L.grid : T.total_chunks;
    if (g <= 0) return cudaSuccess;
    if (g > 0x7fffffffLL) g = 0x7fffffffLL;
    const size_t sm = sgrad_bytes(S);
    k_pprb<<<(int)g, L.block, sm, st>>>(S, P, G, T, counter, status, pers, sigma);
    return cudaGetLastError();
}
cudaError_t pprb_attributes(cudaFuncAttributes* a) {
    return cudaFuncGetAttributes(a, reinterpret_cast<const void*>(&k_pprb));
}
int pprb_occupancy(int block, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void*>(&k_pprb), block, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

}  // namespace dppt
