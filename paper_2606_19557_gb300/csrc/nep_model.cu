// Per-atom kernels of the NEP loss + parameter-gradient pass (hot-path steps a2-a4,
// a6 and a8-a10), one warp per centre atom, persistent over a static species-sorted
// schedule (each warp owns a contiguous range of work positions).
//
// Forward (k_forward):
//   A_nlm = sum_j g^A_n(r_ij) Y_lm(r^_ij)          per-pair geometry staged in shared
//                                                   memory, lanes own (l, m) outputs
//   q_n   = sum_b sum_k c^{t_i b}_{nk} S^b_k,  S^b_k = sum_{j: t_j = b} f_k(r_ij)
//                                                   (the radial descriptor is linear in c)
//   q_nl  = sum_m A_nlm^2, q4_n, q5_n               (Methods, Eq. "q3b"; 4-/5-body forms)
//   E_i   = w1 . tanh(W0 q~ - b0) - b1              (Eq. "ann"), e = dE_i/dq~
//   G_p   = dE_i/dd_p                               pair gradients, written per pair
// Adjoint (k_adjoint), for cotangents fbar = dL/dF, ebar = dL/dE_s, wbar = dL/dW_s:
//   lambda_p = fbar_i - fbar_j - wbar_s d_p
//   dq_i = sum_p (dq_i/dd_p) lambda_p               forward-mode JVP of the descriptors
//   reverse through the network (tanh', tanh'') -> per-atom vectors for the network
//   gradient, and abar = dJ/dq; then dJ/dc for every pair (radial part factorised
//   over species sums, angular part per pair).
// All pair and network arithmetic is FP32 with FP32 accumulation inside an atom.
#include "nep_ctx.cuh"

namespace nep {

template <class S>
struct FwdSm {
    static constexpr int SGS = S::NA | 1;
    float q[S::ND];
    float qt[S::ND];
    float b[S::ND];
    float A[S::NA * L3];
    float Ah[S::NA * L3];
    float G4[S::NA * 5];
    float u[NNMAX];
    float sg[32 * SGS];
    float sY[32 * 25];
};

template <class S>
struct AdjSm {
    static constexpr int SGS = S::NA | 1;
    float qt[S::ND];
    float b[S::ND];
    float ab[S::ND];
    float dq[S::ND];
    float dqt[S::ND];
    float A[S::NA * L3];
    float dA[S::NA * L3];
    float Ah[S::NA * L3];
    float Ab[S::NA * L3];
    float G4[S::NA * 5];
    float H4[S::NA * 5];
    float u[NNMAX];
    float zeta[NNMAX];
    float sg[32 * SGS];
    float sgp[32 * SGS];
    float sY[32 * 25];
    float sP[32 * 25];
};

template <class S>
__host__ __device__ size_t fwd_smem_bytes(int T) {
    return ((sizeof(FwdSm<S>) + sizeof(float) * T * (2 * S::KR + S::NC)) + 15) & ~(size_t)15;
}
template <class S>
__host__ __device__ size_t adj_smem_bytes(int T) {
    return ((sizeof(AdjSm<S>) + sizeof(float) * T * (2 * S::KR + S::NCR + S::NCA + S::NC)) + 15) & ~(size_t)15;
}

// Adds the lane-distributed totals of a reduce_scatter<V> to dst[0..K).
template <int V>
__device__ __forceinline__ void flush_add(float *v, float *dst, int K, int lane) {
    reduce_scatter<V>(v, lane);
    if ((lane & RS<V>::DUP_MASK) == 0) {
        const int base = rs_base<V>(lane);
#pragma unroll
        for (int o = 0; o < RS<V>::OUT; ++o)
            if (base + o < K) dst[base + o] += v[o];
    }
}

// ============================================================================= forward

// VAR selects the register budget: 0 -> at most 128 threads x 3 blocks per SM (168
// registers), 1 -> 256 threads x 2 blocks (128 registers); the autotuner times both.
template <class S, int VAR>
__global__ void __launch_bounds__(VAR == 0 ? 128 : 256, VAR == 0 ? 3 : 2) k_forward(AtomArgs a) {
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int SGS = FwdSm<S>::SGS;
    constexpr int VR = pow2ceil(KR);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const size_t stride = fwd_smem_bytes<S>(a.T) / sizeof(float);
    float *base = smem_raw + wib * stride;
    FwdSm<S> &sm = *reinterpret_cast<FwdSm<S> *>(base);
    float *Sr = base + sizeof(FwdSm<S>) / sizeof(float);  // [T][KR]
    float *beta = Sr + a.T * KR;                            // [T][KR]
    float *cw = beta + a.T * KR;                            // [T][NCR] | [T][NCA] of the current species

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const int T = a.T, NN = a.NN;
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);
    const float *W0 = a.par + po.w0;
    const float *W0T = a.par + po.w0t;
    const float *b0 = a.par + po.b0;
    const float *w1 = a.par + po.w1;
    const float b1 = a.par[po.b1];
    const float *scale = a.par + po.scale;
    int cur_t = -1;

    for (int wi = wbeg; wi < wend; ++wi) {
        const int i = a.work[wi];
        const int ti = a.type[i];
        const int64_t beg = a.nbr_off[i], end = a.nbr_off[i + 1];
        const int64_t endA = beg + a.n_ang[i];
        if (ti != cur_t) {  // species-sorted work: rare
            __syncwarp();
            for (int e = lane; e < T * S::NCR; e += 32) cw[e] = a.par[po.cR + (size_t)ti * T * S::NCR + e];
            for (int e = lane; e < T * S::NCA; e += 32) cw[T * S::NCR + e] = a.par[po.cA + (size_t)ti * T * S::NCA + e];
            cur_t = ti;
            __syncwarp();
        }
        const float *cRi = cw;
        const float *cAi = cw + T * S::NCR;

        // ---------------------------------------------------------------- angular moments A_nlm
        float accA[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) accA[n] = 0.0f;
        for (int64_t c0 = beg; c0 < endA; c0 += 32) {
            const int64_t p = c0 + lane;
            if (p < endA) {
                const float4 pd = a.pair[p];
                const int tj = pair_t(pd);
                const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                const float rinv = __frsqrt_rn(r2);
                const float r = r2 * rinv;
                float f[KA];
                basis_val<KA>(r, a.inv_rcA, f);
                const float *c = cAi + tj * S::NCA;
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    float g = 0.0f;
#pragma unroll
                    for (int k = 0; k < KA; ++k) g += c[n * KA + k] * f[k];
                    sm.sg[lane * SGS + n] = g;
                }
                float Y[L3];
                ylm_val(pd.x * rinv, pd.y * rinv, pd.z * rinv, Y);
#pragma unroll
                for (int lm = 0; lm < L3; ++lm) sm.sY[lane * 25 + lm] = Y[lm];
            }
            __syncwarp();
            const int cnt = (int)min((int64_t)32, endA - c0);
            if (lane < L3) {
                for (int pp = 0; pp < cnt; ++pp) {
                    const float y = sm.sY[pp * 25 + lane];
#pragma unroll
                    for (int n = 0; n < NA; ++n) accA[n] += sm.sg[pp * SGS + n] * y;
                }
            }
            __syncwarp();
        }
        if (lane < L3) {
#pragma unroll
            for (int n = 0; n < NA; ++n) sm.A[n * L3 + lane] = accA[n];
        }

        // ---------------------------------------------------------------- radial species sums S^b_k
        for (int e = lane; e < T * KR; e += 32) Sr[e] = 0.0f;
        __syncwarp();
        {
            float v[VR];
#pragma unroll
            for (int k = 0; k < VR; ++k) v[k] = 0.0f;
            int bcur = -1;
            for (int64_t c0 = beg; c0 < end; c0 += 32) {
                const int64_t p = c0 + lane;
                const bool valid = p < end;
                int tj = -1;
                float f[KR];
#pragma unroll
                for (int k = 0; k < KR; ++k) f[k] = 0.0f;
                if (valid) {
                    const float4 pd = a.pair[p];
                    tj = pair_t(pd);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float r = r2 * __frsqrt_rn(r2);
                    basis_val<KR>(r, a.inv_rcR, f);
                }
                unsigned rem = __ballot_sync(FULL, valid);
                while (rem) {
                    const int leader = __ffs(rem) - 1;
                    const int bsp = __shfl_sync(FULL, tj, leader);
                    const bool inb = valid && tj == bsp;
                    rem &= ~__ballot_sync(FULL, inb);
                    if (bsp != bcur) {
                        if (bcur >= 0) flush_add<VR>(v, Sr + bcur * KR, KR, lane);
#pragma unroll
                        for (int k = 0; k < VR; ++k) v[k] = 0.0f;
                        bcur = bsp;
                    }
                    if (inb) {
#pragma unroll
                        for (int k = 0; k < KR; ++k) v[k] += f[k];
                    }
                }
            }
            if (bcur >= 0) flush_add<VR>(v, Sr + bcur * KR, KR, lane);
        }
        __syncwarp();

        // ---------------------------------------------------------------- descriptors
        if (lane < NR) {
            float q = 0.0f;
            for (int bb = 0; bb < T; ++bb) {
#pragma unroll
                for (int k = 0; k < KR; ++k) q += cRi[bb * S::NCR + lane * KR + k] * Sr[bb * KR + k];
            }
            sm.q[lane] = q;
        }
        for (int e = lane; e < 4 * NA; e += 32) {
            const int n = e % NA, l = e / NA + 1;
            const float *Ar = sm.A + n * L3 + l * l - 1;
            float s = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) s += Ar[m] * Ar[m];
            sm.q[NR + (l - 1) * NA + n] = s;
        }
        if (lane < NA) {
            const float *An = sm.A + lane * L3;
            float Mt[6], M2[6], pr[5];
            l2_matrix(An + 3, Mt);
            sym_prod(Mt, Mt, M2);
            sm.q[NR + 4 * NA + lane] = KAPPA_REAL * sym_trace_prod(M2, Mt);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) sm.G4[lane * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
            const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
            sm.q[NR + 5 * NA + lane] = q1 * q1;
        }
        __syncwarp();
        for (int e = lane; e < ND; e += 32) sm.qt[e] = sm.q[e] * scale[e];
        __syncwarp();

        // ---------------------------------------------------------------- network (Eq. "ann")
        float Epart = 0.0f;
        for (int mu = lane; mu < NN; mu += 32) {
            float z = -b0[ti * NN + mu];
            const float *wt = W0T + (size_t)ti * ND * NN + mu;
#pragma unroll 5
            for (int v = 0; v < ND; ++v) z += wt[(size_t)v * NN] * sm.qt[v];
            const float h = tanhf(z);
            a.st_h[(size_t)wi * NN + mu] = h;
            const float wv = w1[ti * NN + mu];
            Epart += wv * h;
            sm.u[mu] = wv * (1.0f - h * h);
        }
        const float Ei = warp_sum(Epart) - b1;
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            const float *wr = W0 + (size_t)ti * NN * ND + v;
            float e = 0.0f;
            for (int mu = 0; mu < NN; ++mu) e += wr[(size_t)mu * ND] * sm.u[mu];
            sm.b[v] = e * scale[v];
        }
        __syncwarp();

        // ---------------------------------------------------------------- dE_i/dA and radial factors
        if (lane < L3) {
            const int lm = lane, l = l_of_lm(lm);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                const float av = sm.A[n * L3 + lm];
                float ah = 2.0f * sm.b[NR + (l - 1) * NA + n] * av;
                if (l == 2) ah += sm.b[NR + 4 * NA + n] * sm.G4[n * 5 + (lm - 3)];
                if (l == 1) ah += sm.b[NR + 5 * NA + n] * 4.0f * sm.q[NR + n] * av;
                sm.Ah[n * L3 + lm] = ah;
            }
        }
        for (int e = lane; e < T * KR; e += 32) {
            const int bb = e / KR, k = e - bb * KR;
            float s = 0.0f;
#pragma unroll
            for (int n = 0; n < NR; ++n) s += sm.b[n] * cRi[bb * S::NCR + n * KR + k];
            beta[e] = s;
        }
        __syncwarp();

        // ---------------------------------------------------------------- pair gradients, angular part
        float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
        float W9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) W9[k] = 0.0f;
        for (int64_t p = beg + lane; p < endA; p += 32) {
            const float4 pd = a.pair[p];
            const int tj = pair_t(pd);
            const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
            const float rinv = __frsqrt_rn(r2);
            const float r = r2 * rinv;
            const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
            float f[KA], fp[KA];
            basis_val_der<KA>(r, a.inv_rcA, f, fp);
            const float *c = cAi + tj * S::NCA;
            float g[NA], gp[NA];
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                for (int k = 0; k < KA; ++k) {
                    s0 += c[n * KA + k] * f[k];
                    s1 += c[n * KA + k] * fp[k];
                }
                g[n] = s0;
                gp[n] = s1;
            }
            float srad = 0.0f, Vx = 0.0f, Vy = 0.0f, Vz = 0.0f;
            ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float ah = sm.Ah[n * L3 + lm];
                    a1 += ah * g[n];
                    a2 += ah * gp[n];
                }
                srad += a2 * Y;
                Vx += a1 * gx;
                Vy += a1 * gy;
                Vz += a1 * gz;
            });
            const float uv = ux * Vx + uy * Vy + uz * Vz;
            const float Gx = srad * ux + (Vx - ux * uv) * rinv;
            const float Gy = srad * uy + (Vy - uy * uv) * rinv;
            const float Gz = srad * uz + (Vz - uz * uv) * rinv;
            a.G[p] = make_float4(Gx, Gy, Gz, 0.0f);
            Fx += Gx;
            Fy += Gy;
            Fz += Gz;
            W9[0] -= Gx * pd.x; W9[1] -= Gx * pd.y; W9[2] -= Gx * pd.z;
            W9[3] -= Gy * pd.x; W9[4] -= Gy * pd.y; W9[5] -= Gy * pd.z;
            W9[6] -= Gz * pd.x; W9[7] -= Gz * pd.y; W9[8] -= Gz * pd.z;
        }
        // ---------------------------------------------------------------- pair gradients, radial part
        for (int64_t p = beg + lane; p < end; p += 32) {
            const float4 pd = a.pair[p];
            const int tj = pair_t(pd);
            const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
            const float rinv = __frsqrt_rn(r2);
            const float r = r2 * rinv;
            float f[KR], fp[KR];
            basis_val_der<KR>(r, a.inv_rcR, f, fp);
            const float *be = beta + tj * KR;
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < KR; ++k) s += be[k] * fp[k];
            s *= rinv;
            const float Gx = s * pd.x, Gy = s * pd.y, Gz = s * pd.z;
            float4 gt = make_float4(Gx, Gy, Gz, 0.0f);
            if (p < endA) {
                const float4 g0 = a.G[p];  // angular part, written by this lane above
                gt.x += g0.x;
                gt.y += g0.y;
                gt.z += g0.z;
            }
            a.G[p] = gt;
            Fx += Gx;
            Fy += Gy;
            Fz += Gz;
            W9[0] -= Gx * pd.x; W9[1] -= Gx * pd.y; W9[2] -= Gx * pd.z;
            W9[3] -= Gy * pd.x; W9[4] -= Gy * pd.y; W9[5] -= Gy * pd.z;
            W9[6] -= Gz * pd.x; W9[7] -= Gz * pd.y; W9[8] -= Gz * pd.z;
        }
        {
            float v[16] = {Fx, Fy, Fz, W9[0], W9[1], W9[2], W9[3], W9[4], W9[5], W9[6], W9[7], W9[8],
                           0.0f, 0.0f, 0.0f, 0.0f};
            reduce_scatter<16>(v, lane);
            const int idx = rs_base<16>(lane);
            if ((lane & 1) == 0) {
                if (idx < 3) a.F_own[(size_t)i * 3 + idx] = v[0];
                else if (idx < 12) a.W_atom[(size_t)i * 9 + idx - 3] = v[0];
            }
        }
        if (lane == 0) a.E_atom[i] = Ei;
        for (int e = lane; e < ND; e += 32) a.st_qt[(size_t)wi * ND + e] = sm.qt[e];
        for (int e = lane; e < NA * L3; e += 32) a.st_A[(size_t)wi * NA * L3 + e] = sm.A[e];
        if (a.q_raw)
            for (int e = lane; e < ND; e += 32) a.q_raw[(size_t)i * ND + e] = sm.q[e];
        __syncwarp();
    }
}

// ============================================================================= adjoint

template <class S, int VAR>
__global__ void __launch_bounds__(VAR == 0 ? 128 : 256, VAR == 0 ? 3 : 2) k_adjoint(AtomArgs a) {
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int NCR = S::NCR, NCA = S::NCA, NC = S::NC;
    constexpr int SGS = AdjSm<S>::SGS;
    constexpr int VR2 = pow2ceil(2 * KR);
    constexpr int VA = pow2ceil(NCA);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int T = a.T, NN = a.NN;
    const size_t stride = adj_smem_bytes<S>(T) / sizeof(float);
    float *base = smem_raw + wib * stride;
    AdjSm<S> &sm = *reinterpret_cast<AdjSm<S> *>(base);
    float *Sr = base + sizeof(AdjSm<S>) / sizeof(float);  // [T][2 KR]: S^b_k | S'^b_k
    float *accR = Sr + T * 2 * KR;                          // [T][NCR]
    float *accA = accR + T * NCR;                           // [T][NCA]
    float *cw = accA + T * NCA;                             // [T][NCR] | [T][NCA] of the current species

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);
    const float *W0 = a.par + po.w0;
    const float *W0T = a.par + po.w0t;
    const float *w1 = a.par + po.w1;
    const float *scale = a.par + po.scale;

    int cur_t = -1;
    auto flush_slot = [&](int t) {
        float *dst = a.cpart + (size_t)(w + t) * T * NC;
        for (int bb = 0; bb < T; ++bb) {
            for (int e = lane; e < NCR; e += 32) dst[(size_t)bb * NC + e] = accR[bb * NCR + e];
            for (int e = lane; e < NCA; e += 32) dst[(size_t)bb * NC + NCR + e] = accA[bb * NCA + e];
        }
    };

    for (int wi = wbeg; wi < wend; ++wi) {
        const int i = a.work[wi];
        const int ti = a.type[i];
        if (ti != cur_t) {
            __syncwarp();
            if (cur_t >= 0) flush_slot(cur_t);
            for (int e = lane; e < T * NCR; e += 32) accR[e] = 0.0f;
            for (int e = lane; e < T * NCA; e += 32) accA[e] = 0.0f;
            for (int e = lane; e < T * NCR; e += 32) cw[e] = a.par[po.cR + (size_t)ti * T * NCR + e];
            for (int e = lane; e < T * NCA; e += 32) cw[T * NCR + e] = a.par[po.cA + (size_t)ti * T * NCA + e];
            cur_t = ti;
            __syncwarp();
        }
        const int s = a.struct_of[i];
        const int64_t beg = a.nbr_off[i], end = a.nbr_off[i + 1];
        const int64_t endA = beg + a.n_ang[i];
        const float *cRi = cw;
        const float *cAi = cw + T * NCR;

        // ---------------------------------------------------------------- state of the forward pass
        for (int e = lane; e < ND; e += 32) sm.qt[e] = a.st_qt[(size_t)wi * ND + e];
        for (int e = lane; e < NA * L3; e += 32) sm.A[e] = a.st_A[(size_t)wi * NA * L3 + e];
        float hreg[NNMAX / 32];
#pragma unroll
        for (int k = 0; k < NNMAX / 32; ++k) {
            const int mu = lane + 32 * k;
            hreg[k] = 0.0f;
            if (mu < NN) {
                const float h = a.st_h[(size_t)wi * NN + mu];
                hreg[k] = h;
                sm.u[mu] = w1[ti * NN + mu] * (1.0f - h * h);
            }
        }
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            const float *wr = W0 + (size_t)ti * NN * ND + v;
            float e = 0.0f;
            for (int mu = 0; mu < NN; ++mu) e += wr[(size_t)mu * ND] * sm.u[mu];
            sm.b[v] = e * scale[v];
        }
        if (lane < NA) {
            const float *An = sm.A + lane * L3;
            float Mt[6], M2[6], pr[5];
            l2_matrix(An + 3, Mt);
            sym_prod(Mt, Mt, M2);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) sm.G4[lane * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
        }
        __syncwarp();
        if (lane < L3) {
            const int lm = lane, l = l_of_lm(lm);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                const float *An = sm.A + n * L3;
                const float av = An[lm];
                float ah = 2.0f * sm.b[NR + (l - 1) * NA + n] * av;
                if (l == 2) ah += sm.b[NR + 4 * NA + n] * sm.G4[n * 5 + (lm - 3)];
                if (l == 1) {
                    const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
                    ah += sm.b[NR + 5 * NA + n] * 4.0f * q1 * av;
                }
                sm.Ah[n * L3 + lm] = ah;
            }
        }
        const float fbx = a.fbar[(size_t)i * 3], fby = a.fbar[(size_t)i * 3 + 1], fbz = a.fbar[(size_t)i * 3 + 2];
        float Wb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Wb[k] = a.wbar[(size_t)s * 9 + k];
        const float eb = a.ebar[s];
        __syncwarp();

        // ---------------------------------------------------------------- angular JVP: dA_nlm
        float accd[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) accd[n] = 0.0f;
        for (int64_t c0 = beg; c0 < endA; c0 += 32) {
            const int64_t p = c0 + lane;
            if (p < endA) {
                const float4 pd = a.pair[p];
                const int j = pair_j(pd), tj = pair_t(pd);
                const float lx = fbx - a.fbar[(size_t)j * 3] - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                const float ly = fby - a.fbar[(size_t)j * 3 + 1] - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                const float lz = fbz - a.fbar[(size_t)j * 3 + 2] - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                const float rinv = __frsqrt_rn(r2);
                const float r = r2 * rinv;
                const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
                const float rl = ux * lx + uy * ly + uz * lz;
                const float px = (lx - rl * ux) * rinv, py = (ly - rl * uy) * rinv, pz = (lz - rl * uz) * rinv;
                float f[KA], fp[KA];
                basis_val_der<KA>(r, a.inv_rcA, f, fp);
                const float *c = cAi + tj * NCA;
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        s0 += c[n * KA + k] * f[k];
                        s1 += c[n * KA + k] * fp[k];
                    }
                    sm.sg[lane * SGS + n] = s0;
                    sm.sgp[lane * SGS + n] = s1 * rl;
                }
                ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                    sm.sY[lane * 25 + lm] = Y;
                    sm.sP[lane * 25 + lm] = gx * px + gy * py + gz * pz;
                });
            }
            __syncwarp();
            const int cnt = (int)min((int64_t)32, endA - c0);
            if (lane < L3) {
                for (int pp = 0; pp < cnt; ++pp) {
                    const float y = sm.sY[pp * 25 + lane], ps = sm.sP[pp * 25 + lane];
#pragma unroll
                    for (int n = 0; n < NA; ++n) accd[n] += sm.sgp[pp * SGS + n] * y + sm.sg[pp * SGS + n] * ps;
                }
            }
            __syncwarp();
        }
        if (lane < L3) {
#pragma unroll
            for (int n = 0; n < NA; ++n) sm.dA[n * L3 + lane] = accd[n];
        }

        // ---------------------------------------------------------------- radial JVP species sums
        for (int e = lane; e < T * 2 * KR; e += 32) Sr[e] = 0.0f;
        __syncwarp();
        {
            float v[VR2];
#pragma unroll
            for (int k = 0; k < VR2; ++k) v[k] = 0.0f;
            int bcur = -1;
            for (int64_t c0 = beg; c0 < end; c0 += 32) {
                const int64_t p = c0 + lane;
                const bool valid = p < end;
                int tj = -1;
                float f[KR], fp[KR];
#pragma unroll
                for (int k = 0; k < KR; ++k) f[k] = fp[k] = 0.0f;
                float rl = 0.0f;
                if (valid) {
                    const float4 pd = a.pair[p];
                    const int j = pair_j(pd);
                    tj = pair_t(pd);
                    const float lx = fbx - a.fbar[(size_t)j * 3] - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                    const float ly = fby - a.fbar[(size_t)j * 3 + 1] - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                    const float lz = fbz - a.fbar[(size_t)j * 3 + 2] - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = __frsqrt_rn(r2);
                    const float r = r2 * rinv;
                    rl = (pd.x * lx + pd.y * ly + pd.z * lz) * rinv;
                    basis_val_der<KR>(r, a.inv_rcR, f, fp);
                }
                unsigned rem = __ballot_sync(FULL, valid);
                while (rem) {
                    const int leader = __ffs(rem) - 1;
                    const int bsp = __shfl_sync(FULL, tj, leader);
                    const bool inb = valid && tj == bsp;
                    rem &= ~__ballot_sync(FULL, inb);
                    if (bsp != bcur) {
                        if (bcur >= 0) flush_add<VR2>(v, Sr + bcur * 2 * KR, 2 * KR, lane);
#pragma unroll
                        for (int k = 0; k < VR2; ++k) v[k] = 0.0f;
                        bcur = bsp;
                    }
                    if (inb) {
#pragma unroll
                        for (int k = 0; k < KR; ++k) {
                            v[k] += f[k];
                            v[KR + k] += rl * fp[k];
                        }
                    }
                }
            }
            if (bcur >= 0) flush_add<VR2>(v, Sr + bcur * 2 * KR, 2 * KR, lane);
        }
        __syncwarp();

        // ---------------------------------------------------------------- JVP of the descriptors
        if (lane < NR) {
            float d = 0.0f;
            for (int bb = 0; bb < T; ++bb) {
#pragma unroll
                for (int k = 0; k < KR; ++k) d += cRi[bb * NCR + lane * KR + k] * Sr[bb * 2 * KR + KR + k];
            }
            sm.dq[lane] = d;
        }
        for (int e = lane; e < 4 * NA; e += 32) {
            const int n = e % NA, l = e / NA + 1;
            const float *Ar = sm.A + n * L3 + l * l - 1;
            const float *dAr = sm.dA + n * L3 + l * l - 1;
            float s2 = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) s2 += Ar[m] * dAr[m];
            sm.dq[NR + (l - 1) * NA + n] = 2.0f * s2;
        }
        if (lane < NA) {
            const float *An = sm.A + lane * L3;
            const float *dAn = sm.dA + lane * L3;
            float d4 = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) d4 += sm.G4[lane * 5 + m] * dAn[3 + m];
            sm.dq[NR + 4 * NA + lane] = d4;
            float Mt[6], dMt[6], P[6], pr[5];
            l2_matrix(An + 3, Mt);
            l2_matrix(dAn + 3, dMt);
            sym_prod(Mt, dMt, P);
            l2_project(P, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) sm.H4[lane * 5 + m] = 6.0f * KAPPA_REAL * pr[m];
            const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
            const float ad = An[0] * dAn[0] + An[1] * dAn[1] + An[2] * dAn[2];
            sm.dq[NR + 5 * NA + lane] = 4.0f * q1 * ad;
        }
        __syncwarp();
        for (int e = lane; e < ND; e += 32) sm.dqt[e] = sm.dq[e] * scale[e];
        __syncwarp();

        // ---------------------------------------------------------------- reverse through the network
#pragma unroll
        for (int k = 0; k < NNMAX / 32; ++k) {
            const int mu = lane + 32 * k;
            if (mu < NN) {
                float v = 0.0f;
                const float *wt = W0T + (size_t)ti * ND * NN + mu;
#pragma unroll 5
                for (int q = 0; q < ND; ++q) v += wt[(size_t)q * NN] * sm.dqt[q];
                const float h = hreg[k];
                const float hp = 1.0f - h * h;
                const float hpp = -2.0f * h * hp;
                const float wv = w1[ti * NN + mu];
                const float ze = eb * wv * hp + wv * hpp * v;
                sm.zeta[mu] = ze;
                a.zt[(size_t)wi * NN + mu] = ze;
                a.ut[(size_t)wi * NN + mu] = wv * hp;
                a.om[(size_t)wi * NN + mu] = eb * h + hp * v;
            }
        }
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            const float *wr = W0 + (size_t)ti * NN * ND + v;
            float e = 0.0f;
            for (int mu = 0; mu < NN; ++mu) e += wr[(size_t)mu * ND] * sm.zeta[mu];
            sm.ab[v] = e * scale[v];
            a.dqt[(size_t)wi * ND + v] = sm.dqt[v];
        }
        __syncwarp();

        // ---------------------------------------------------------------- dJ/dA
        if (lane < L3) {
            const int lm = lane, l = l_of_lm(lm);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                const float *An = sm.A + n * L3;
                const float *dAn = sm.dA + n * L3;
                const int v3 = NR + (l - 1) * NA + n;
                float x = 2.0f * sm.ab[v3] * An[lm] + 2.0f * sm.b[v3] * dAn[lm];
                if (l == 2) x += sm.ab[NR + 4 * NA + n] * sm.G4[n * 5 + lm - 3] + sm.b[NR + 4 * NA + n] * sm.H4[n * 5 + lm - 3];
                if (l == 1) {
                    const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
                    const float ad = An[0] * dAn[0] + An[1] * dAn[1] + An[2] * dAn[2];
                    const int v5 = NR + 5 * NA + n;
                    x += sm.ab[v5] * 4.0f * q1 * An[lm] + sm.b[v5] * (8.0f * ad * An[lm] + 4.0f * q1 * dAn[lm]);
                }
                sm.Ab[n * L3 + lm] = x;
            }
        }
        // ---------------------------------------------------------------- radial coefficient gradient
        for (int e = lane; e < T * NCR; e += 32) {
            const int bb = e / NCR, rr = e - bb * NCR, n = rr / KR, k = rr - n * KR;
            accR[e] += sm.ab[n] * Sr[bb * 2 * KR + k] + sm.b[n] * Sr[bb * 2 * KR + KR + k];
        }
        __syncwarp();

        // ---------------------------------------------------------------- angular coefficient gradient
        {
            float X[VA];
#pragma unroll
            for (int e = 0; e < VA; ++e) X[e] = 0.0f;
            int bcur = -1;
            for (int64_t c0 = beg; c0 < endA; c0 += 32) {
                const int64_t p = c0 + lane;
                const bool valid = p < endA;
                int tj = -1;
                float f[KA], fp[KA], al[NA], be[NA];
#pragma unroll
                for (int k = 0; k < KA; ++k) f[k] = fp[k] = 0.0f;
#pragma unroll
                for (int n = 0; n < NA; ++n) al[n] = be[n] = 0.0f;
                if (valid) {
                    const float4 pd = a.pair[p];
                    const int j = pair_j(pd);
                    tj = pair_t(pd);
                    const float lx = fbx - a.fbar[(size_t)j * 3] - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                    const float ly = fby - a.fbar[(size_t)j * 3 + 1] - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                    const float lz = fbz - a.fbar[(size_t)j * 3 + 2] - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = __frsqrt_rn(r2);
                    const float r = r2 * rinv;
                    const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
                    const float rl = ux * lx + uy * ly + uz * lz;
                    const float px = (lx - rl * ux) * rinv, py = (ly - rl * uy) * rinv, pz = (lz - rl * uz) * rinv;
                    basis_val_der<KA>(r, a.inv_rcA, f, fp);
                    ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                        const float ps = gx * px + gy * py + gz * pz;
#pragma unroll
                        for (int n = 0; n < NA; ++n) {
                            const float ah = sm.Ah[n * L3 + lm];
                            al[n] += sm.Ab[n * L3 + lm] * Y + ah * ps;
                            be[n] += ah * Y;
                        }
                    });
#pragma unroll
                    for (int n = 0; n < NA; ++n) be[n] *= rl;
                }
                unsigned rem = __ballot_sync(FULL, valid);
                while (rem) {
                    const int leader = __ffs(rem) - 1;
                    const int bsp = __shfl_sync(FULL, tj, leader);
                    const bool inb = valid && tj == bsp;
                    rem &= ~__ballot_sync(FULL, inb);
                    if (bsp != bcur) {
                        if (bcur >= 0) flush_add<VA>(X, accA + bcur * NCA, NCA, lane);
#pragma unroll
                        for (int e = 0; e < VA; ++e) X[e] = 0.0f;
                        bcur = bsp;
                    }
                    if (inb) {
#pragma unroll
                        for (int n = 0; n < NA; ++n)
#pragma unroll
                            for (int k = 0; k < KA; ++k) X[n * KA + k] += al[n] * f[k] + be[n] * fp[k];
                    }
                }
            }
            if (bcur >= 0) flush_add<VA>(X, accA + bcur * NCA, NCA, lane);
        }
        __syncwarp();
    }
    __syncwarp();
    if (cur_t >= 0) flush_slot(cur_t);
}

// ============================================================================= dispatch

template <class S, int VAR>
void launch_fwd_t(const AtomArgs &a, int blocks, int wpb, size_t smem, cudaStream_t st) {
    k_forward<S, VAR><<<blocks, wpb * 32, smem, st>>>(a);
}
template <class S, int VAR>
void launch_adj_t(const AtomArgs &a, int blocks, int wpb, size_t smem, cudaStream_t st) {
    k_adjoint<S, VAR><<<blocks, wpb * 32, smem, st>>>(a);
}

template <int NR, int KR, int NA, int KA>
KernelSet make_set() {
    using S = Shape<NR, KR, NA, KA>;
    KernelSet k;
    k.NR = NR;
    k.KR = KR;
    k.NA = NA;
    k.KA = KA;
    k.fwd_fn[0] = (const void *)k_forward<S, 0>;
    k.fwd_fn[1] = (const void *)k_forward<S, 1>;
    k.adj_fn[0] = (const void *)k_adjoint<S, 0>;
    k.adj_fn[1] = (const void *)k_adjoint<S, 1>;
    k.max_wpb[0] = 4;
    k.max_wpb[1] = 8;
    k.fwd_smem = fwd_smem_bytes<S>;
    k.adj_smem = adj_smem_bytes<S>;
    k.launch_fwd[0] = launch_fwd_t<S, 0>;
    k.launch_fwd[1] = launch_fwd_t<S, 1>;
    k.launch_adj[0] = launch_adj_t<S, 0>;
    k.launch_adj[1] = launch_adj_t<S, 1>;
    return k;
}

static const KernelSet g_sets[] = {
    make_set<5, 9, 5, 9>(),      // n_max 4/4, basis 8/8 (the 16-element NEPOri/NEP44 shape)
    make_set<7, 11, 7, 11>(),    // n_max 6/6, basis 10/10
    make_set<12, 12, 12, 12>(),  // any shape within the limits
};

const KernelSet *select_kernels(int nR, int kR, int nA, int kA) {
    for (const KernelSet &k : g_sets)
        if (nR <= k.NR && kR <= k.KR && nA <= k.NA && kA <= k.KA) return &k;
    return nullptr;
}

}  // namespace nep
