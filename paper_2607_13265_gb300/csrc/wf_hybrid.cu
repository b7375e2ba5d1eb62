// Hybrid cached replay (Sec. 4.4, Eq. hybrid_decision) in the wavefront schedule.  The
// traversal kernels are the wavefront's own; these kernels replace its cache pass and its
// replay.  Each runs the hybrid visitor of the megakernel (hybrid.cuh) on one path per
// thread, its per-path arrays bound to the path's records in the workspace:
//   cache pass (one vertex per iteration): the block emission e_b and throughput T_b of the
//     vertex's block, the vertex's route per channel (scalar PRB, inversion or
//     recomputation), and at the path's end the backward fold over the blocks that leaves
//     the suffixes L[c_b] at the checkpoints and the path's value (the primal runs this pass
//     alone, so that its waves need no per-vertex cache either);
//   replay (one vertex per iteration): when a block with a recomputed vertex starts, its
//     vertices are shaded again, detached, from their cached hits (no ray is traced twice)
//     and folded onto the next checkpoint's suffix; then the vertex is replayed with dual
//     numbers, L[v+1] taken from a checkpoint, by its route, or from that look-ahead.
// All material types share one replay kernel (no binning).
#include "wavefront.cuh"
#include "hybrid.cuh"

namespace dppt {

template <int K>
__device__ __forceinline__ void hyb_bind(HybVis<128, K>& vis, const HybWs& H, int q, int cap) {
    vis.ck = reinterpret_cast<float (*)[60]>(H.ck + (long long)q * H.nb * 60);
    vis.route = H.route + (long long)q * H.rstride;
    vis.blk = reinterpret_cast<float (*)[31]>(H.blk + (long long)q * K * 31);
    vis.bt = H.btr + (long long)q * 60;
    vis.ebr = vis.bt + 48;
    vis.flags = H.flags + (long long)q * H.fw;
    vis.gamma = H.gamma;
    vis.eps = H.eps;
    vis.cap = cap;
}

template <int PHASE, int K, bool NM>
__global__ void __launch_bounds__(128, 2)
k_wf_hyb(const DScene S, const DParams P, const DGrads G, const __grid_constant__ JobTable T, WfState W, WfLists L,
         HybWs H) {
    extern __shared__ float sgrad[];
    if (PHASE == 1) sgrad_zero(S, sgrad);
    const int* list = PHASE == 0 ? L.l0 : L.bins + (long long)kBinOther * L.binQ;
    const int count = PHASE == 0 ? L.cur[0] : L.cur[8 + kBinOther];
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += stride) {
        const int q = list[idx];
        const WfMeta m = W.path[q].meta;
        const DJob& J = T.job[m.job];
        const unsigned long long pid = (unsigned long long)m.lo | ((unsigned long long)m.hi << 32);
        Walk w;
        get_walk(W.path + q, w);
        HybVis<128, K> vis;
        vis.S = &S; vis.P = &P; vis.G = &G; vis.sgrad = sgrad;
        hyb_bind<K>(vis, H, q, W.cap);
        vis.n = (m.pni >> 8) & 0xff; vis.i = (m.pni >> 16) & 0xff; vis.phase = PHASE;
        vis.la = 0; vis.blk_base = 0;
        VCtx vc;
        NeePending ne;
        Shade sh;
        bool cont = false, done = false;
        int phase = PHASE;
        if (PHASE == 0) {
            if (vis.n == 0)
                for (int k = 0; k < H.fw; ++k) vis.flags[k] = 0u;
            if (get_vertex(W.vtx + q, w, vc, ne, sh)) {
                if (NM) apply_normal_map(S, P, vc);
                const int visible = W.visible[q];
                const int slot = w.v - 1;
                cont = walk_finish(S, P, w, vc, ne, visible != 0, sh, vis);
                H.vis[(long long)slot * W.Q + q] = visible != 0 ? 1 : 0;
            }
            if (cont) {
                L.next0[atomicAdd(L.nxt + 0, 1)] = q;
            } else {
                float L0[12];
                vis.fold(L0);
                Rot<float> Rc = camera_rot(S.cams[J.cam], w.d1);
                const float inv = 1.0f / (float)J.spp;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v[4] = {L0[4 * c], L0[4 * c + 1], L0[4 * c + 2], L0[4 * c + 3]};
                    rot_apply(Rc, v);
                    W.raw[3 * (long long)q + c] = make_float4(v[0] * inv, v[1] * inv, v[2] * inv, v[3] * inv);
                }
                if (vis.n > 0 && J.dS) {     // the adjoint (a primal job has no image adjoint)
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
                    bin_append(L, kBinOther, q);
                } else {
                    done = true;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 r = W.path[q].arow[c];
                vis.a[c][0] = r.x; vis.a[c][1] = r.y; vis.a[c][2] = r.z; vis.a[c][3] = r.w;
            }
            if (vis.i < vis.n && vis.i % K == 0 && vis.flagged(vis.i / K)) {
                // the block again, detached, from its cached hits up to the next checkpoint
                Walk w2 = w;
                vis.phase = 2; vis.la = 0; vis.blk_base = vis.i;
                while (vis.la < K && w2.v - 1 < W.cap) {
                    const int slot = w2.v - 1;
                    const float4 hv = *reinterpret_cast<const float4*>(W.hit_rec(slot, q));
                    if (__float_as_int(hv.w) == kMissCode) break;
                    HitRec h;
                    decode_hit(S, hv, h);
                    VCtx vc2;
                    NeePending ne2;
                    Shade sh2;
                    walk_shade<NM>(S, P, J, pid, w2, h, vc2, ne2, sh2);
                    if (!walk_finish(S, P, w2, vc2, ne2, H.vis[(long long)slot * W.Q + q] != 0, sh2, vis)) break;
                }
                vis.fold_block();
                vis.phase = 1;
            }
            const int slot = w.v - 1;
            const float4 hv = *reinterpret_cast<const float4*>(W.hit_rec(slot, q));
            if (__float_as_int(hv.w) != kMissCode) {
                HitRec h;
                decode_hit(S, hv, h);
                walk_shade<NM>(S, P, J, pid, w, h, vc, ne, sh);
                cont = walk_finish(S, P, w, vc, ne, H.vis[(long long)slot * W.Q + q] != 0, sh, vis);
            }
            // the replay goes on while the next ray found a vertex
            if (cont && w.v - 1 < W.cap &&
                __float_as_int(reinterpret_cast<const float4*>(W.hit_rec(w.v - 1, q))->w) != kMissCode)
                bin_append(L, kBinOther, q);
            else
                done = true;
            if (!done) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    W.path[q].arow[c] = make_float4(vis.a[c][0], vis.a[c][1], vis.a[c][2], vis.a[c][3]);
            }
        }
        if (done) {
            if (J.sig) J.sig[pid] = fnv(w.sig, (unsigned)w.nv);
        } else {
            W.path[q].meta.pni = phase | (vis.n << 8) | (vis.i << 16);
            put_walk(W.path + q, w);
        }
    }
    if (PHASE == 1) sgrad_flush(S, G, sgrad);
}

// (compiled with the normal-map code: the hybrid is the memory-saving replay, not the fast one)
template <int K>
static cudaError_t launch_k(int phase, const DScene& S, const DParams& P, const DGrads& G, const JobTable& T,
                            const WfState& W, const WfLists& L, const HybWs& H, int grid, size_t smem, cudaStream_t st) {
    if (phase == 0) k_wf_hyb<0, K, true><<<grid, 128, 0, st>>>(S, P, G, T, W, L, H);
    else k_wf_hyb<1, K, true><<<grid, 128, smem, st>>>(S, P, G, T, W, L, H);
    return cudaGetLastError();
}

cudaError_t launch_wf_hybrid(int phase, int K, const DScene& S, const DParams& P, const DGrads& G,
                             const JobTable& T, const WfState& W, const WfLists& L, const HybWs& H, int grid,
                             size_t smem, cudaStream_t st) {
    switch (K) {
        case 4: return launch_k<4>(phase, S, P, G, T, W, L, H, grid, smem, st);
        case 8: return launch_k<8>(phase, S, P, G, T, W, L, H, grid, smem, st);
        case 16: return launch_k<16>(phase, S, P, G, T, W, L, H, grid, smem, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dppt
