// Camera-filter folds for batches of polarizer angles: the filter does not
// change the paths, so the raw sensor-frame image is rendered once and each
// angle's image, the adjoint input and the angle gradients are per-pixel maps.
#include <algorithm>

#include "device_math.cuh"
#include "internal.h"

namespace dppt {

// ================================================================== camera-filter folds
// C(theta) for the filter stacks, in the sensor frame (c = cos 2theta, s = sin 2theta):
// polarizer  1/2 [[1,c,s,0],[c,c^2,cs,0],[s,cs,s^2,0],[0,0,0,0]];
// quarter-wave plate (fast axis x) then polarizer: columns (0,1,3) as above with the
// s-column moved to the circular slot.
__device__ __forceinline__ void filter_matrix(int filter, float theta, float C[16], float dC[16]) {
    float s, c;
    sincosf(2.0f * theta, &s, &c);
    float P[16] = {0.5f, 0.5f * c, 0.5f * s, 0.0f,
                   0.5f * c, 0.5f * c * c, 0.5f * c * s, 0.0f,
                   0.5f * s, 0.5f * c * s, 0.5f * s * s, 0.0f,
                   0.0f, 0.0f, 0.0f, 0.0f};
    // d/dtheta with dc = -2s, ds = 2c
    float dP[16] = {0.0f, -s, c, 0.0f,
                    -s, -2.0f * c * s, c * c - s * s, 0.0f,
                    c, c * c - s * s, 2.0f * s * c, 0.0f,
                    0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = 0; r < 4; ++r) {
        if (filter == DPPT_FILTER_POLARIZER) {
            for (int k = 0; k < 4; ++k) { C[4 * r + k] = P[4 * r + k]; dC[4 * r + k] = dP[4 * r + k]; }
        } else {  // P . Q(pi/2, 0): column 2 <- -column 3 (= 0), column 3 <- column 2
            C[4 * r + 0] = P[4 * r + 0]; C[4 * r + 1] = P[4 * r + 1]; C[4 * r + 2] = -P[4 * r + 3]; C[4 * r + 3] = P[4 * r + 2];
            dC[4 * r + 0] = dP[4 * r + 0]; dC[4 * r + 1] = dP[4 * r + 1]; dC[4 * r + 2] = -dP[4 * r + 3]; dC[4 * r + 3] = dP[4 * r + 2];
        }
    }
}

// Every job of a call in one launch: each block belongs to one job (the jobs' blocks back to
// back, block0[j] the first of job j), so that the small images of a batch, which cannot fill
// the GPU alone, run side by side instead of one launch after another.
struct FoldBatch {
    FoldJob job[kMaxFoldJobs];
    int block0[kMaxFoldJobs + 1];
    int njobs;
};
__device__ __forceinline__ int fold_job_of_block(const FoldBatch& b) {
    int lo = 0, hi = b.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.block0[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// image[a][pix] = C(theta_a) raw[pix] of every filtered job
__global__ void k_apply_filter(const __grid_constant__ FoldBatch b) {
    extern __shared__ float sC[];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    for (int a = threadIdx.x; a < J.nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_matrix(J.filter, __ldg(J.theta + a), C, dC);
        for (int k = 0; k < 16; ++k) sC[16 * a + k] = C[k];
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    if (pix >= J.npix) return;
    float r[12];
    const float4* rp = reinterpret_cast<const float4*>(J.raw + pix * 12);
    for (int q = 0; q < 3; ++q) { float4 t = __ldg(rp + q); r[4 * q] = t.x; r[4 * q + 1] = t.y; r[4 * q + 2] = t.z; r[4 * q + 3] = t.w; }
    for (int a = 0; a < J.nang; ++a) {
        const float* C = sC + 16 * a;
        float4* op = reinterpret_cast<float4*>(J.image + ((long long)a * J.npix + pix) * 12);
        for (int c = 0; c < 3; ++c) {
            const float* v = r + 4 * c;
            float o[4];
            for (int i = 0; i < 4; ++i) o[i] = C[4 * i] * v[0] + C[4 * i + 1] * v[1] + C[4 * i + 2] * v[2] + C[4 * i + 3] * v[3];
            op[c] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

// dS[pix] = sum_a C_a^T dI_a[pix] of every filtered job
__global__ void k_filter_adjoint_input(const __grid_constant__ FoldBatch b) {
    extern __shared__ float sC[];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    for (int a = threadIdx.x; a < J.nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_matrix(J.filter, __ldg(J.theta + a), C, dC);
        for (int k = 0; k < 16; ++k) sC[16 * a + k] = C[k];
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    if (pix >= J.npix) return;
    float acc[12];
    for (int k = 0; k < 12; ++k) acc[k] = 0.0f;
    for (int a = 0; a < J.nang; ++a) {
        const float* C = sC + 16 * a;
        const float4* dp = reinterpret_cast<const float4*>(J.dimage + ((long long)a * J.npix + pix) * 12);
        for (int c = 0; c < 3; ++c) {
            float4 t = __ldg(dp + c);
            float g[4] = {t.x, t.y, t.z, t.w};
            for (int j = 0; j < 4; ++j)
                acc[4 * c + j] += C[j] * g[0] + C[4 + j] * g[1] + C[8 + j] * g[2] + C[12 + j] * g[3];
        }
    }
    float4* o = reinterpret_cast<float4*>(J.dS + pix * 12);
    for (int q = 0; q < 3; ++q) o[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// dtheta_a += sum_pix dI_a[pix]^T dC_a/dtheta S_adj[pix] of every filtered job
__global__ void k_theta_grad(const __grid_constant__ FoldBatch b) {
    extern __shared__ float sm[];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    const int nang = J.nang;
    float* sdC = sm;               // [nang][16]
    float* sacc = sm + 16 * nang;  // [nang]
    for (int a = threadIdx.x; a < nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_matrix(J.filter, __ldg(J.theta + a), C, dC);
        for (int k = 0; k < 16; ++k) sdC[16 * a + k] = dC[k];
        sacc[a] = 0.0f;
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    const bool act = pix < J.npix;     // every lane takes part in the warp sums below
    float s[12];
    for (int k = 0; k < 12; ++k) s[k] = 0.0f;
    if (act) {
        const float4* sp = reinterpret_cast<const float4*>(J.S_adj + pix * 12);
        for (int q = 0; q < 3; ++q) { float4 t = __ldg(sp + q); s[4 * q] = t.x; s[4 * q + 1] = t.y; s[4 * q + 2] = t.z; s[4 * q + 3] = t.w; }
    }
    for (int a = 0; a < nang; ++a) {
        float v = 0.0f;
        if (act) {
            const float* dC = sdC + 16 * a;
            const float4* dp = reinterpret_cast<const float4*>(J.dimage + ((long long)a * J.npix + pix) * 12);
            for (int c = 0; c < 3; ++c) {
                float4 t = __ldg(dp + c);
                float g[4] = {t.x, t.y, t.z, t.w};
                for (int i = 0; i < 4; ++i)
                    v += g[i] * (dC[4 * i] * s[4 * c] + dC[4 * i + 1] * s[4 * c + 1] + dC[4 * i + 2] * s[4 * c + 2] + dC[4 * i + 3] * s[4 * c + 3]);
            }
        }
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v != 0.0f) atomicAdd(sacc + a, v);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < nang; a += blockDim.x)
        if (sacc[a] != 0.0f) atomicAdd(J.dtheta + a, sacc[a]);
}

// ================================================================== fused L2 loss folds
// The loss scale * sum_a sum_pix |C_a raw - T_a|^2 of a job and its derivatives, with the
// residual C_a raw - T_a formed per pixel and never stored (raw [pix][12], target in the
// image layout [a][pix][12]).  An unfiltered job (filter none) has one "angle" with C = I.
__device__ __forceinline__ void load12(const float* p, float v[12]) {
    const float4* q = reinterpret_cast<const float4*>(p);
    for (int k = 0; k < 3; ++k) { float4 t = __ldg(q + k); v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w; }
}
__device__ __forceinline__ void filter_or_identity(int filter, const float* theta, int a, float C[16], float dC[16]) {
    if (filter == DPPT_FILTER_NONE) {
        for (int k = 0; k < 16; ++k) { C[k] = (k % 5 == 0) ? 1.0f : 0.0f; dC[k] = 0.0f; }
    } else {
        filter_matrix(filter, __ldg(theta + a), C, dC);
    }
}
// residual of channel c at angle a: d = C v - t
__device__ __forceinline__ void residual4(const float* C, const float* v, const float* t, float d[4]) {
    for (int i = 0; i < 4; ++i) d[i] = C[4 * i] * v[0] + C[4 * i + 1] * v[1] + C[4 * i + 2] * v[2] + C[4 * i + 3] * v[3] - t[i];
}

// scale * sum_a sum_pix |C_a raw - T_a|^2 of every job, added into *loss
__global__ void k_l2_loss(const __grid_constant__ FoldBatch b, double scale, double* loss) {
    extern __shared__ float sC[];
    __shared__ double swarp[32];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    for (int a = threadIdx.x; a < J.nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_or_identity(J.filter, J.theta, a, C, dC);
        for (int k = 0; k < 16; ++k) sC[16 * a + k] = C[k];
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (pix < J.npix) {
        float r[12], t[12];
        load12(J.raw + pix * 12, r);
        float part = 0.0f;
        for (int a = 0; a < J.nang; ++a) {
            load12(J.target + ((long long)a * J.npix + pix) * 12, t);
            for (int c = 0; c < 3; ++c) {
                float d[4];
                residual4(sC + 16 * a, r + 4 * c, t + 4 * c, d);
                part += d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3];
            }
        }
        acc = (double)part;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += swarp[w];
        if (s != 0.0) atomicAdd(loss, s * scale);
    }
}

// dS = 2 scale sum_a C_a^T (C_a raw - T_a) of every job
__global__ void k_l2_adjoint_input(const __grid_constant__ FoldBatch b, float scale2) {
    extern __shared__ float sC[];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    for (int a = threadIdx.x; a < J.nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_or_identity(J.filter, J.theta, a, C, dC);
        for (int k = 0; k < 16; ++k) sC[16 * a + k] = C[k];
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    if (pix >= J.npix) return;
    float r[12], t[12], acc[12];
    load12(J.raw + pix * 12, r);
    for (int k = 0; k < 12; ++k) acc[k] = 0.0f;
    for (int a = 0; a < J.nang; ++a) {
        const float* C = sC + 16 * a;
        load12(J.target + ((long long)a * J.npix + pix) * 12, t);
        for (int c = 0; c < 3; ++c) {
            float d[4];
            residual4(C, r + 4 * c, t + 4 * c, d);
            for (int j = 0; j < 4; ++j)
                acc[4 * c + j] += C[j] * d[0] + C[4 + j] * d[1] + C[8 + j] * d[2] + C[12 + j] * d[3];
        }
    }
    float4* o = reinterpret_cast<float4*>(J.dS + pix * 12);
    for (int q = 0; q < 3; ++q)
        o[q] = make_float4(scale2 * acc[4 * q], scale2 * acc[4 * q + 1], scale2 * acc[4 * q + 2], scale2 * acc[4 * q + 3]);
}

// dtheta_a += 2 scale sum_pix (C_a raw - T_a)^T dC_a S_adj of every (filtered) job
__global__ void k_l2_theta_grad(const __grid_constant__ FoldBatch b, float scale2) {
    extern __shared__ float sm[];
    const int jb = fold_job_of_block(b);
    const FoldJob& J = b.job[jb];
    const int nang = J.nang;
    float* sC = sm;                 // [nang][16]
    float* sdC = sm + 16 * nang;    // [nang][16]
    float* sacc = sm + 32 * nang;   // [nang]
    for (int a = threadIdx.x; a < nang; a += blockDim.x) {
        float C[16], dC[16];
        filter_matrix(J.filter, __ldg(J.theta + a), C, dC);
        for (int k = 0; k < 16; ++k) { sC[16 * a + k] = C[k]; sdC[16 * a + k] = dC[k]; }
        sacc[a] = 0.0f;
    }
    __syncthreads();
    const long long pix = (long long)(blockIdx.x - b.block0[jb]) * blockDim.x + threadIdx.x;
    const bool act = pix < J.npix;     // every lane takes part in the warp sums below
    float r[12], s[12], t[12];
    for (int k = 0; k < 12; ++k) { r[k] = 0.0f; s[k] = 0.0f; }
    if (act) { load12(J.raw + pix * 12, r); load12(J.S_adj + pix * 12, s); }
    for (int a = 0; a < nang; ++a) {
        float v = 0.0f;
        if (act) {
            load12(J.target + ((long long)a * J.npix + pix) * 12, t);
            const float* dC = sdC + 16 * a;
            for (int c = 0; c < 3; ++c) {
                float d[4];
                residual4(sC + 16 * a, r + 4 * c, t + 4 * c, d);
                for (int i = 0; i < 4; ++i)
                    v += d[i] * (dC[4 * i] * s[4 * c] + dC[4 * i + 1] * s[4 * c + 1] + dC[4 * i + 2] * s[4 * c + 2] +
                                 dC[4 * i + 3] * s[4 * c + 3]);
            }
        }
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v != 0.0f) atomicAdd(sacc + a, v * scale2);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < nang; a += blockDim.x)
        if (sacc[a] != 0.0f) atomicAdd(J.dtheta + a, sacc[a]);
}

// The batched folds: the jobs in chunks of kMaxFoldJobs, one launch per chunk, 256 threads
// per block, one pixel per thread.  smem_per_angle: floats of shared memory per angle.
template <class Launch>
static cudaError_t launch_fold_batches(const FoldJob* jobs, int njobs, int smem_per_angle, const void* kernel,
                                       Launch launch) {
    constexpr int kBlock = 256;
    for (int j0 = 0; j0 < njobs; j0 += kMaxFoldJobs) {
        FoldBatch b{};
        b.njobs = std::min(kMaxFoldJobs, njobs - j0);
        long long blocks = 0;
        int nang = 1;
        for (int k = 0; k < b.njobs; ++k) {
            b.job[k] = jobs[j0 + k];
            b.block0[k] = (int)blocks;
            blocks += (b.job[k].npix + kBlock - 1) / kBlock;
            nang = std::max(nang, b.job[k].nang);
        }
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        b.block0[b.njobs] = (int)blocks;
        if (blocks == 0) continue;
        const size_t smem = sizeof(float) * (size_t)smem_per_angle * nang;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        launch(b, (int)blocks, kBlock, smem);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
int fold_launches(int njobs) { return (njobs + kMaxFoldJobs - 1) / kMaxFoldJobs; }
cudaError_t launch_apply_filter(const FoldJob* jobs, int njobs, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 16, reinterpret_cast<const void*>(&k_apply_filter),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) { k_apply_filter<<<g, blk, sm, st>>>(b); });
}
cudaError_t launch_filter_adjoint_input(const FoldJob* jobs, int njobs, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 16, reinterpret_cast<const void*>(&k_filter_adjoint_input),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) {
                                   k_filter_adjoint_input<<<g, blk, sm, st>>>(b);
                               });
}
cudaError_t launch_theta_grad(const FoldJob* jobs, int njobs, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 17, reinterpret_cast<const void*>(&k_theta_grad),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) { k_theta_grad<<<g, blk, sm, st>>>(b); });
}
cudaError_t launch_l2_loss(const FoldJob* jobs, int njobs, double scale, double* loss, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 16, reinterpret_cast<const void*>(&k_l2_loss),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) {
                                   k_l2_loss<<<g, blk, sm, st>>>(b, scale, loss);
                               });
}
cudaError_t launch_l2_adjoint_input(const FoldJob* jobs, int njobs, float scale2, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 16, reinterpret_cast<const void*>(&k_l2_adjoint_input),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) {
                                   k_l2_adjoint_input<<<g, blk, sm, st>>>(b, scale2);
                               });
}
cudaError_t launch_l2_theta_grad(const FoldJob* jobs, int njobs, float scale2, cudaStream_t st) {
    return launch_fold_batches(jobs, njobs, 33, reinterpret_cast<const void*>(&k_l2_theta_grad),
                               [&](const FoldBatch& b, int g, int blk, size_t sm) {
                                   k_l2_theta_grad<<<g, blk, sm, st>>>(b, scale2);
                               });
}

}  // namespace dppt
