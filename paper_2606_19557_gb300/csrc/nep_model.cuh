// Per-atom kernels of the NEP loss + parameter-gradient pass (hot-path steps a2-a4, a6,
// a8-a10).  Persistent over a static species-sorted schedule: each warp owns a
// contiguous range of work positions and processes them in batches of G = 32/SW
// atoms of one species, one group of SW lanes per atom, so that the ~15-20 angular
// and ~60-80 radial neighbours of an atom keep most lanes busy.
//
// Forward (k_forward):
//   A_nlm = sum_j g^A_n(r_ij) Y_lm(r^_ij)          pair geometry staged in shared memory,
//                                                   lanes own (l, m) outputs
//   q_n   = sum_b sum_k c^{t_i b}_{nk} S^b_k,  S^b_k = sum_{j: t_j = b} f_k(r_ij)
//                                                   (the radial descriptor is linear in c)
//   q_nl  = sum_m A_nlm^2, q4_n, q5_n               (Methods, Eq. "q3b"; 4-/5-body readings)
//   E_i   = w1 . tanh(W0 q~ - b0) - b1              (Eq. "ann"), e = dE_i/dq~
//   G_p   = dE_i/dd_p                               pair gradients, written per pair
// Adjoint (k_adjoint), for cotangents fbar = dL/dF, ebar = dL/dE_s, wbar = dL/dW_s:
//   lambda_p = fbar_i - fbar_j - wbar_s d_p
//   dq_i = sum_p (dq_i/dd_p) lambda_p               forward-mode JVP of the descriptors
//   reverse through the network (tanh', tanh'') -> per-atom vectors for the network
//   gradient, abar = dJ/dq; then dJ/dc (radial part factorised over species sums,
//   angular part per pair).
// FP32 arithmetic with FP32 accumulation inside an atom; no floating-point atomics:
// species runs of different groups are flushed into the warp's accumulators one group
// after the other, so results are bit-reproducible for a fixed launch shape.
#pragma once

#include "nep_ctx.cuh"

namespace nep {

// ============================================================================= layouts

template <class S, int SW>
struct FwdL {
    static constexpr int G = 32 / SW;
    static constexpr int SGS = (S::NA + 3) & ~3;  // rows of g_n padded to float4
    static constexpr int NLMO = (L3 + SW - 1) / SW;  // (l, m) outputs owned per lane
    struct Atom {
        float q[S::ND];
        float qt[S::ND];
        float b[S::ND];
        float A[S::NA * L3];
        float Ah[S::NA * L3];
        float G4[S::NA * 5];
    };
    Atom at[G];
    __align__(16) float sg[G][SW][SGS];
    float sY[G][SW][25];
    // runtime tail (floats): u[G][NN], Sr[G][T][KR], beta[G][T][KR], cw[T][NC]
    __host__ __device__ static size_t tail(int T, int NN) {
        return (size_t)G * NN + 2 * (size_t)G * T * S::KR + (size_t)T * S::NC;
    }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(FwdL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

template <class S, int SW>
struct AdjL {
    static constexpr int G = 32 / SW;
    static constexpr int SGS = (S::NA + 3) & ~3;
    static constexpr int NLMO = (L3 + SW - 1) / SW;
    struct Atom {
        float b[S::ND];
        float ab[S::ND];
        float dqt[S::ND];
        float A[S::NA * L3];
        float dA[S::NA * L3];  // dA, then dJ/dA in place
        float Ah[S::NA * L3];
        float G4[S::NA * 5];
        float H4[S::NA * 5];
        float ad[S::NA];  // sum_m A_n1m dA_n1m (read by every l = 1 lane before dA is overwritten)
    };
    Atom at[G];
    __align__(16) float sg[G][SW][SGS];
    __align__(16) float sgp[G][SW][SGS];
    float sY[G][SW][25];
    float sP[G][SW][25];
    // runtime tail: u[G][NN], Sr[G][T][2 KR], accR[T][NCR], accA[T][NCA], cw[T][NC]
    __host__ __device__ static size_t tail(int T, int NN) {
        return (size_t)G * NN + 2 * (size_t)G * T * S::KR + (size_t)T * (S::NCR + S::NCA) + (size_t)T * S::NC;
    }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(AdjL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

// Loads a padded row of N floats (N a multiple of 4, 16-byte aligned) from shared memory.
template <int N>
__device__ __forceinline__ void load_row(const float *src, float *dst) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 t = s4[q];
        dst[4 * q] = t.x;
        dst[4 * q + 1] = t.y;
        dst[4 * q + 2] = t.z;
        dst[4 * q + 3] = t.w;
    }
}

// Batch of up to G = 32/SW consecutive work positions of one species, starting at `base`
// (< wend): group g reads position base + g, so the loads of all groups are in flight
// together.  Returns the species ti, the batch size nb and this group's atom i (the
// batch's first atom for groups beyond nb).
template <int SW>
__device__ __forceinline__ void load_batch(const AtomArgs &a, int base, int wend, int lane, int &ti, int &nb,
                                           int &i) {
    constexpr int G = 32 / SW;
    const int grp = lane / SW;
    const int q = base + grp;
    const int iq = (grp < G && q < wend) ? a.work[q] : -1;
    const int tq = iq >= 0 ? a.type[iq] : -1;
    ti = __shfl_sync(FULL, tq, 0);
    const unsigned same = __ballot_sync(FULL, tq == ti);
    unsigned gm = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) gm |= ((same >> (g * SW)) & 1u) << g;
    nb = min(G, __ffs(~gm) - 1);
    const int i0 = __shfl_sync(FULL, iq, 0);
    i = grp < nb ? iq : i0;
}

// Reduce-scatter the V-vector of every group and add the totals of group `grp` into
// dst[0..K) (dst may be shared by the groups: they add one after the other).
template <int V, int SW>
__device__ __forceinline__ void flush_groups(float *v, float *dst, int K, bool has, int lane, bool shared_dst) {
    group_reduce_scatter<V, SW>(v, lane);
    const bool owner = has && ((lane & GRS<V, SW>::DUP_MASK) == 0);
    const int base = grs_base<V, SW>(lane);
    if (!shared_dst) {
        if (owner) {
#pragma unroll
            for (int o = 0; o < GRS<V, SW>::OUT; ++o)
                if (base + o < K) dst[base + o] += v[o];
        }
    } else {
        const int grp = lane / SW;
#pragma unroll 1
        for (int g = 0; g < 32 / SW; ++g) {
            if (grp == g && owner) {
#pragma unroll
                for (int o = 0; o < GRS<V, SW>::OUT; ++o)
                    if (base + o < K) dst[base + o] += v[o];
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = 0.0f;
}

// ============================================================================= forward

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(VAR == 0 ? 128 : 256, VAR == 0 ? 3 : 2) k_forward(AtomArgs a) {
    using L = FwdL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int G = L::G, SGS = L::SGS, NLMO = L::NLMO;
    constexpr int VR = pow2ceil(KR);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *tail = base_ptr + sizeof(L) / sizeof(float);
    float *Sr = tail + G * NN + grp * T * KR;                // [T][KR] of this group
    float *beta = tail + G * NN + G * T * KR + grp * T * KR; // [T][KR] of this group
    float *cw = tail + G * NN + 2 * G * T * KR;              // [T][NCR] | [T][NCA], current species

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);
    const float *W0 = a.par + po.w0;
    const float *W0T = a.par + po.w0t;
    const float *b0 = a.par + po.b0;
    const float *w1 = a.par + po.w1;
    const float b1 = a.par[po.b1];
    const float *scale = a.par + po.scale;
    int cur_t = -1;

    for (int bp = wbeg; bp < wend;) {
        int ti, nb, i;
        load_batch<SW>(a, bp, wend, lane, ti, nb, i);
        const bool act = grp < nb;
        const int bp0 = bp;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
        if (ti != cur_t) {  // species-sorted work: rare
            __syncwarp();
            for (int e = lane; e < T * S::NCR; e += 32) cw[e] = a.par[po.cR + (size_t)ti * T * S::NCR + e];
            for (int e = lane; e < T * S::NCA; e += 32) cw[T * S::NCR + e] = a.par[po.cA + (size_t)ti * T * S::NCA + e];
            cur_t = ti;
            __syncwarp();
        }
        const float *cRi = cw;
        const float *cAi = cw + T * S::NCR;
        const int64_t beg = a.nbr_off[i];
        const int nRad = act ? (int)(a.nbr_off[i + 1] - beg) : 0;
        const int nAng = act ? a.n_ang[i] : 0;
        const int maxR = __reduce_max_sync(FULL, nRad);
        const int maxA = __reduce_max_sync(FULL, nAng);
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their pair records into L2
            const int ni = a.work[bp + grp];
            const int64_t nb0 = a.nbr_off[ni], nb1 = a.nbr_off[ni + 1];
            prefetch_l2(a.pair + nb0, sizeof(float4) * (size_t)(nb1 - nb0), sl, SW);
        }

        // ---------------------------------------------------------------- angular moments A_nlm
        float accA[NLMO][NA];
#pragma unroll
        for (int j = 0; j < NLMO; ++j)
#pragma unroll
            for (int n = 0; n < NA; ++n) accA[j][n] = 0.0f;
        const float4 *prs = a.pair + beg;
        float4 nxt = pair_or_zero(prs, sl, nAng);
        for (int c0 = 0; c0 < maxA; c0 += SW) {
            const int k = c0 + sl;
            const float4 pd = nxt;
            nxt = pair_or_zero(prs, k + SW, nAng);
            if (k < nAng) {
                const int tj = pair_t(pd);
                const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                const float rinv = inv_norm(r2);
                const float r = r2 * rinv;
                float f[KA];
                basis_val<KA>(r, a.inv_rcA, f);
                const float *c = cAi + tj * S::NCA;
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    float g = 0.0f;
#pragma unroll
                    for (int kk = 0; kk < KA; ++kk) g += c[n * KA + kk] * f[kk];
                    sm.sg[grp][sl][n] = g;
                }
                float Y[L3];
                ylm_val(pd.x * rinv, pd.y * rinv, pd.z * rinv, Y);
#pragma unroll
                for (int lm = 0; lm < L3; ++lm) sm.sY[grp][sl][lm] = Y[lm];
            }
            __syncwarp();
            const int cnt = min(SW, nAng - c0);
            for (int pp = 0; pp < cnt; ++pp) {
                float gv[SGS];
                load_row<SGS>(sm.sg[grp][pp], gv);
#pragma unroll
                for (int j = 0; j < NLMO; ++j) {
                    const int lm = sl + j * SW;
                    if (lm < L3) {
                        const float y = sm.sY[grp][pp][lm];
#pragma unroll
                        for (int n = 0; n < NA; ++n) accA[j][n] += gv[n] * y;
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < NLMO; ++j) {
            const int lm = sl + j * SW;
            if (lm < L3) {
#pragma unroll
                for (int n = 0; n < NA; ++n) at.A[n * L3 + lm] = accA[j][n];
            }
        }

        // ---------------------------------------------------------------- radial species sums S^b_k
        for (int e = sl; e < T * KR; e += SW) Sr[e] = 0.0f;
        __syncwarp();
        {
            float v[VR];
#pragma unroll
            for (int k = 0; k < VR; ++k) v[k] = 0.0f;
            int bcur = -1;
            float4 nxr = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const bool valid = k < nRad;
                const float4 pd = nxr;
                nxr = pair_or_zero(prs, k + SW, nRad);
                int tj = -1;
                float f[KR];
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) f[kk] = 0.0f;
                if (valid) {
                    tj = pair_t(pd);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    basis_val<KR>(r2 * inv_norm(r2), a.inv_rcR, f);
                }
                if (T == 1) {  // one species: no runs to track
                    if (valid) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) v[kk] += f[kk];
                    }
                    continue;
                }
                unsigned rem = group_bits<SW>(__ballot_sync(FULL, valid), lane);
                while (__any_sync(FULL, rem != 0)) {
                    const bool has = rem != 0;
                    const int leader = has ? __ffs(rem) - 1 : 0;
                    int bsp = __shfl_sync(FULL, tj, (lane & ~(SW - 1)) + leader);
                    if (!has) bsp = bcur;
                    const bool inb = valid && has && tj == bsp;
                    rem &= ~group_bits<SW>(__ballot_sync(FULL, inb), lane);
                    const bool change = bsp != bcur;
                    if (__any_sync(FULL, change && bcur >= 0))
                        flush_groups<VR, SW>(v, Sr + (bcur >= 0 ? bcur : 0) * KR, KR, bcur >= 0, lane, false);
                    bcur = bsp;
                    if (inb) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) v[kk] += f[kk];
                    }
                }
            }
            if (T == 1 && nRad > 0) bcur = 0;
            if (__any_sync(FULL, bcur >= 0)) flush_groups<VR, SW>(v, Sr + (bcur >= 0 ? bcur : 0) * KR, KR, bcur >= 0, lane, false);
        }
        __syncwarp();

        // ---------------------------------------------------------------- descriptors
        for (int n = sl; n < NR; n += SW) {
            float q = 0.0f;
            for (int bb = 0; bb < T; ++bb) {
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) q += cRi[bb * S::NCR + n * KR + kk] * Sr[bb * KR + kk];
            }
            at.q[n] = q;
        }
        for (int e = sl; e < 4 * NA; e += SW) {
            const int n = e % NA, l = e / NA + 1;
            const float *Ar = at.A + n * L3 + l * l - 1;
            float s2 = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) s2 += Ar[m] * Ar[m];
            at.q[NR + (l - 1) * NA + n] = s2;
        }
        for (int n = sl; n < NA; n += SW) {
            const float *An = at.A + n * L3;
            float Mt[6], M2[6], pr[5];
            l2_matrix(An + 3, Mt);
            sym_prod(Mt, Mt, M2);
            at.q[NR + 4 * NA + n] = KAPPA_REAL * sym_trace_prod(M2, Mt);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.G4[n * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
            const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
            at.q[NR + 5 * NA + n] = q1 * q1;
        }
        __syncwarp();
        for (int e = sl; e < ND; e += SW) at.qt[e] = at.q[e] * scale[e];
        __syncwarp();

        // ---------------------------------------------------------------- network (Eq. "ann")
        // The G atoms of the batch share the species, so the layer runs as a small
        // batched product: lanes index neurons (then descriptor components) and each
        // weight is loaded once for all G atoms.
        float Eg[G];
#pragma unroll
        for (int g = 0; g < G; ++g) Eg[g] = 0.0f;
        for (int mu = lane; mu < NN; mu += 32) {
            float z[G];
            const float bz = -b0[ti * NN + mu];
#pragma unroll
            for (int g = 0; g < G; ++g) z[g] = bz;
            const float *wt = W0T + (size_t)ti * ND * NN + mu;
#pragma unroll
            for (int v = 0; v < ND; ++v) {
                const float wv = wt[(size_t)v * NN];
#pragma unroll
                for (int g = 0; g < G; ++g) z[g] += wv * sm.at[g].qt[v];
            }
            const float wo = w1[ti * NN + mu];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float h = tanhf(z[g]);
                if (g < nb) a.st_h[(size_t)(bp0 + g) * NN + mu] = h;
                Eg[g] += wo * h;
                tail[g * NN + mu] = wo * (1.0f - h * h);  // u of atom g
            }
        }
        float Ei = 0.0f;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float e = warp_sum(Eg[g]);
            if (g == grp) Ei = e - b1;
        }
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            float e[G];
#pragma unroll
            for (int g = 0; g < G; ++g) e[g] = 0.0f;
            const float *wr = W0 + (size_t)ti * NN * ND + v;
#pragma unroll 10
            for (int mu = 0; mu < NN; ++mu) {
                const float wv = wr[(size_t)mu * ND];
#pragma unroll
                for (int g = 0; g < G; ++g) e[g] += wv * tail[g * NN + mu];
            }
            const float sc = scale[v];
#pragma unroll
            for (int g = 0; g < G; ++g) sm.at[g].b[v] = e[g] * sc;
        }
        __syncwarp();

        // ---------------------------------------------------------------- dE_i/dA and radial factors
#pragma unroll
        for (int j = 0; j < NLMO; ++j) {
            const int lm = sl + j * SW;
            if (lm < L3) {
                const int l = l_of_lm(lm);
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float av = at.A[n * L3 + lm];
                    float ah = 2.0f * at.b[NR + (l - 1) * NA + n] * av;
                    if (l == 2) ah += at.b[NR + 4 * NA + n] * at.G4[n * 5 + (lm - 3)];
                    if (l == 1) ah += at.b[NR + 5 * NA + n] * 4.0f * at.q[NR + n] * av;
                    at.Ah[n * L3 + lm] = ah;
                }
            }
        }
        for (int e = sl; e < T * KR; e += SW) {
            const int bb = e / KR, kk = e - bb * KR;
            float s2 = 0.0f;
#pragma unroll
            for (int n = 0; n < NR; ++n) s2 += at.b[n] * cRi[bb * S::NCR + n * KR + kk];
            beta[e] = s2;
        }
        __syncwarp();

        // ---------------------------------------------------------------- pair gradients
        float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
        float W9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) W9[k] = 0.0f;
        // angular neighbours: angular and radial parts of G_p together
        float4 nxf = pair_or_zero(prs, sl, nAng);
        for (int k = sl; k < nAng; k += SW) {
            const int64_t p = beg + k;
            const float4 pd = nxf;
            nxf = pair_or_zero(prs, k + SW, nAng);
            const int tj = pair_t(pd);
            const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
            const float rinv = inv_norm(r2);
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
                for (int kk = 0; kk < KA; ++kk) {
                    s0 += c[n * KA + kk] * f[kk];
                    s1 += c[n * KA + kk] * fp[kk];
                }
                g[n] = s0;
                gp[n] = s1;
            }
            float srad = 0.0f, Vx = 0.0f, Vy = 0.0f, Vz = 0.0f;
            ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float ah = at.Ah[n * L3 + lm];
                    a1 += ah * g[n];
                    a2 += ah * gp[n];
                }
                srad += a2 * Y;
                Vx += a1 * gx;
                Vy += a1 * gy;
                Vz += a1 * gz;
            });
            {
                float fr[KR], fpr[KR];
                basis_val_der<KR>(r, a.inv_rcR, fr, fpr);
                const float *be = beta + tj * KR;
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) srad += be[kk] * fpr[kk];
            }
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
        // radial-only neighbours
        nxf = pair_or_zero(prs, nAng + sl, nRad);
        for (int k = nAng + sl; k < nRad; k += SW) {
            const int64_t p = beg + k;
            const float4 pd = nxf;
            nxf = pair_or_zero(prs, k + SW, nRad);
            const int tj = pair_t(pd);
            const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
            const float rinv = inv_norm(r2);
            float f[KR], fp[KR];
            basis_val_der<KR>(r2 * rinv, a.inv_rcR, f, fp);
            const float *be = beta + tj * KR;
            float s2 = 0.0f;
#pragma unroll
            for (int kk = 0; kk < KR; ++kk) s2 += be[kk] * fp[kk];
            s2 *= rinv;
            const float Gx = s2 * pd.x, Gy = s2 * pd.y, Gz = s2 * pd.z;
            a.G[p] = make_float4(Gx, Gy, Gz, 0.0f);
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
            group_reduce_scatter<16, SW>(v, lane);
            const int base = grs_base<16, SW>(lane);
            if (act && (lane & GRS<16, SW>::DUP_MASK) == 0) {
#pragma unroll
                for (int o = 0; o < GRS<16, SW>::OUT; ++o) {
                    const int idx = base + o;
                    if (idx < 3) a.F_own[(size_t)i * 3 + idx] = v[o];
                    else if (idx < 12) a.W_atom[(size_t)i * 9 + idx - 3] = v[o];
                }
            }
        }
        if (act) {
            if (sl == 0) a.E_atom[i] = Ei;
            for (int e = sl; e < ND; e += SW) a.st_qt[(size_t)wi * ND + e] = at.qt[e];
            for (int e = sl; e < NA * L3; e += SW) a.st_A[(size_t)wi * NA * L3 + e] = at.A[e];
            if (a.q_raw)
                for (int e = sl; e < ND; e += SW) a.q_raw[(size_t)i * ND + e] = at.q[e];
        }
        __syncwarp();
    }
}

// ============================================================================= adjoint

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(VAR == 0 ? 128 : 256, VAR == 0 ? 3 : 2) k_adjoint(AtomArgs a) {
    using L = AdjL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int NCR = S::NCR, NCA = S::NCA, NC = S::NC;
    constexpr int G = L::G, NLMO = L::NLMO;
    constexpr int VR2 = pow2ceil(2 * KR);
    constexpr int VA = pow2ceil(NCA);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *tail = base_ptr + sizeof(L) / sizeof(float);
    float *Sr = tail + G * NN + grp * T * 2 * KR;         // [T][2 KR] S^b_k | S'^b_k of this group
    float *accR = tail + G * NN + G * T * 2 * KR;         // [T][NCR] (warp)
    float *accA = accR + T * NCR;                         // [T][NCA] (warp)
    float *cw = accA + T * NCA;                           // [T][NCR] | [T][NCA], current species

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

    for (int bp = wbeg; bp < wend;) {
        int ti, nb, i;
        load_batch<SW>(a, bp, wend, lane, ti, nb, i);
        const bool act = grp < nb;
        const int bp0 = bp;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
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
        const float *cRi = cw;
        const float *cAi = cw + T * NCR;
        const int s = a.struct_of[i];
        const int64_t beg = a.nbr_off[i];
        const int nRad = act ? (int)(a.nbr_off[i + 1] - beg) : 0;
        const int nAng = act ? a.n_ang[i] : 0;
        const int maxR = __reduce_max_sync(FULL, nRad);
        const int maxA = __reduce_max_sync(FULL, nAng);
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their pair records into L2
            const int ni = a.work[bp + grp];
            const int64_t nb0 = a.nbr_off[ni], nb1 = a.nbr_off[ni + 1];
            prefetch_l2(a.pair + nb0, sizeof(float4) * (size_t)(nb1 - nb0), sl, SW);
        }

        // ---------------------------------------------------------------- state of the forward pass
#pragma unroll
        for (int e = sl; e < NA * L3; e += SW) at.A[e] = a.st_A[(size_t)wi * NA * L3 + e];
        for (int mu = lane; mu < NN; mu += 32) {
            const float wo = w1[ti * NN + mu];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float h = a.st_h[(size_t)(bp0 + (g < nb ? g : 0)) * NN + mu];
                tail[g * NN + mu] = wo * (1.0f - h * h);
            }
        }
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            float e[G];
#pragma unroll
            for (int g = 0; g < G; ++g) e[g] = 0.0f;
            const float *wr = W0 + (size_t)ti * NN * ND + v;
#pragma unroll 10
            for (int mu = 0; mu < NN; ++mu) {
                const float wv = wr[(size_t)mu * ND];
#pragma unroll
                for (int g = 0; g < G; ++g) e[g] += wv * tail[g * NN + mu];
            }
            const float sc = scale[v];
#pragma unroll
            for (int g = 0; g < G; ++g) sm.at[g].b[v] = e[g] * sc;
        }
        for (int n = sl; n < NA; n += SW) {
            const float *An = at.A + n * L3;
            float Mt[6], M2[6], pr[5];
            l2_matrix(An + 3, Mt);
            sym_prod(Mt, Mt, M2);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.G4[n * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NLMO; ++j) {
            const int lm = sl + j * SW;
            if (lm < L3) {
                const int l = l_of_lm(lm);
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float *An = at.A + n * L3;
                    const float av = An[lm];
                    float ah = 2.0f * at.b[NR + (l - 1) * NA + n] * av;
                    if (l == 2) ah += at.b[NR + 4 * NA + n] * at.G4[n * 5 + (lm - 3)];
                    if (l == 1) {
                        const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
                        ah += at.b[NR + 5 * NA + n] * 4.0f * q1 * av;
                    }
                    at.Ah[n * L3 + lm] = ah;
                }
            }
        }
        const float4 *prs = a.pair + beg;
        const float4 fbi = a.fbar[i];
        const float fbx = fbi.x, fby = fbi.y, fbz = fbi.z;
        float Wb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Wb[k] = a.wbar[(size_t)s * 9 + k];
        const float eb = a.ebar[s];
        __syncwarp();

        // ---------------------------------------------------------------- angular JVP: dA_nlm
        {
            float accd[NLMO][NA];
#pragma unroll
            for (int j = 0; j < NLMO; ++j)
#pragma unroll
                for (int n = 0; n < NA; ++n) accd[j][n] = 0.0f;
            float4 nxt = pair_or_zero(prs, sl, nAng);
            for (int c0 = 0; c0 < maxA; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nAng);
                if (k < nAng) {
                    const int j = pair_j(pd), tj = pair_t(pd);
                    const float4 fbj = a.fbar[j];
                    const float lx = fbx - fbj.x - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                    const float ly = fby - fbj.y - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                    const float lz = fbz - fbj.z - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
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
                        for (int kk = 0; kk < KA; ++kk) {
                            s0 += c[n * KA + kk] * f[kk];
                            s1 += c[n * KA + kk] * fp[kk];
                        }
                        sm.sg[grp][sl][n] = s0;
                        sm.sgp[grp][sl][n] = s1 * rl;
                    }
                    ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                        sm.sY[grp][sl][lm] = Y;
                        sm.sP[grp][sl][lm] = gx * px + gy * py + gz * pz;
                    });
                }
                __syncwarp();
                const int cnt = min(SW, nAng - c0);
                for (int pp = 0; pp < cnt; ++pp) {
                    float gv[L::SGS], gpv[L::SGS];
                    load_row<L::SGS>(sm.sg[grp][pp], gv);
                    load_row<L::SGS>(sm.sgp[grp][pp], gpv);
#pragma unroll
                    for (int jj = 0; jj < NLMO; ++jj) {
                        const int lm = sl + jj * SW;
                        if (lm < L3) {
                            const float y = sm.sY[grp][pp][lm], ps = sm.sP[grp][pp][lm];
#pragma unroll
                            for (int n = 0; n < NA; ++n) accd[jj][n] += gpv[n] * y + gv[n] * ps;
                        }
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int jj = 0; jj < NLMO; ++jj) {
                const int lm = sl + jj * SW;
                if (lm < L3) {
#pragma unroll
                    for (int n = 0; n < NA; ++n) at.dA[n * L3 + lm] = accd[jj][n];
                }
            }
        }

        // ---------------------------------------------------------------- radial JVP species sums
        for (int e = sl; e < T * 2 * KR; e += SW) Sr[e] = 0.0f;
        __syncwarp();
        {
            float v[VR2];
#pragma unroll
            for (int k = 0; k < VR2; ++k) v[k] = 0.0f;
            int bcur = -1;
            float4 nxt = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const bool valid = k < nRad;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nRad);
                int tj = -1;
                float f[KR], fp[KR];
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) f[kk] = fp[kk] = 0.0f;
                float rl = 0.0f;
                if (valid) {
                    const int j = pair_j(pd);
                    tj = pair_t(pd);
                    const float4 fbj = a.fbar[j];
                    const float lx = fbx - fbj.x - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                    const float ly = fby - fbj.y - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                    const float lz = fbz - fbj.z - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    rl = (pd.x * lx + pd.y * ly + pd.z * lz) * rinv;
                    basis_val_der<KR>(r2 * rinv, a.inv_rcR, f, fp);
                }
                if (T == 1) {  // one species: no runs to track
                    if (valid) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            v[kk] += f[kk];
                            v[KR + kk] += rl * fp[kk];
                        }
                    }
                    continue;
                }
                unsigned rem = group_bits<SW>(__ballot_sync(FULL, valid), lane);
                while (__any_sync(FULL, rem != 0)) {
                    const bool has = rem != 0;
                    const int leader = has ? __ffs(rem) - 1 : 0;
                    int bsp = __shfl_sync(FULL, tj, (lane & ~(SW - 1)) + leader);
                    if (!has) bsp = bcur;
                    const bool inb = valid && has && tj == bsp;
                    rem &= ~group_bits<SW>(__ballot_sync(FULL, inb), lane);
                    const bool change = bsp != bcur;
                    if (__any_sync(FULL, change && bcur >= 0))
                        flush_groups<VR2, SW>(v, Sr + (bcur >= 0 ? bcur : 0) * 2 * KR, 2 * KR, bcur >= 0, lane, false);
                    bcur = bsp;
                    if (inb) {
#pragma unroll
                        for (int kk = 0; kk < KR; ++kk) {
                            v[kk] += f[kk];
                            v[KR + kk] += rl * fp[kk];
                        }
                    }
                }
            }
            if (T == 1 && nRad > 0) bcur = 0;
            if (__any_sync(FULL, bcur >= 0))
                flush_groups<VR2, SW>(v, Sr + (bcur >= 0 ? bcur : 0) * 2 * KR, 2 * KR, bcur >= 0, lane, false);
        }
        __syncwarp();

        // ---------------------------------------------------------------- JVP of the descriptors
        for (int n = sl; n < NR; n += SW) {
            float d = 0.0f;
            for (int bb = 0; bb < T; ++bb) {
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) d += cRi[bb * NCR + n * KR + kk] * Sr[bb * 2 * KR + KR + kk];
            }
            at.dqt[n] = d * scale[n];
        }
        for (int e = sl; e < 4 * NA; e += SW) {
            const int n = e % NA, l = e / NA + 1;
            const float *Ar = at.A + n * L3 + l * l - 1;
            const float *dAr = at.dA + n * L3 + l * l - 1;
            float s2 = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) s2 += Ar[m] * dAr[m];
            const int v = NR + (l - 1) * NA + n;
            at.dqt[v] = 2.0f * s2 * scale[v];
        }
        for (int n = sl; n < NA; n += SW) {
            const float *An = at.A + n * L3;
            const float *dAn = at.dA + n * L3;
            float d4 = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) d4 += at.G4[n * 5 + m] * dAn[3 + m];
            at.dqt[NR + 4 * NA + n] = d4 * scale[NR + 4 * NA + n];
            float Mt[6], dMt[6], Pm[6], pr[5];
            l2_matrix(An + 3, Mt);
            l2_matrix(dAn + 3, dMt);
            sym_prod(Mt, dMt, Pm);
            l2_project(Pm, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.H4[n * 5 + m] = 6.0f * KAPPA_REAL * pr[m];
            const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
            const float ad = An[0] * dAn[0] + An[1] * dAn[1] + An[2] * dAn[2];
            at.ad[n] = ad;
            at.dqt[NR + 5 * NA + n] = 4.0f * q1 * ad * scale[NR + 5 * NA + n];
        }
        __syncwarp();

        // ---------------------------------------------------------------- reverse through the network
        // ebar of every atom of the batch (one structure per atom)
        float ebg[G];
#pragma unroll
        for (int g = 0; g < G; ++g) ebg[g] = __shfl_sync(FULL, eb, g * SW);
        for (int mu = lane; mu < NN; mu += 32) {
            float v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) v[g] = 0.0f;
            const float *wt = W0T + (size_t)ti * ND * NN + mu;
#pragma unroll
            for (int q = 0; q < ND; ++q) {
                const float wv = wt[(size_t)q * NN];
#pragma unroll
                for (int g = 0; g < G; ++g) v[g] += wv * sm.at[g].dqt[q];
            }
            const float wo = w1[ti * NN + mu];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int wg = bp0 + (g < nb ? g : 0);
                const float h = a.st_h[(size_t)wg * NN + mu];
                const float hp = 1.0f - h * h;
                const float hpp = -2.0f * h * hp;
                const float ze = ebg[g] * wo * hp + wo * hpp * v[g];
                tail[g * NN + mu] = ze;  // zeta of atom g
                if (g < nb) {
                    a.zt[(size_t)wg * NN + mu] = ze;
                    a.ut[(size_t)wg * NN + mu] = wo * hp;
                    a.om[(size_t)wg * NN + mu] = ebg[g] * h + hp * v[g];
                }
            }
        }
        __syncwarp();
        for (int v = lane; v < ND; v += 32) {
            float e[G];
#pragma unroll
            for (int g = 0; g < G; ++g) e[g] = 0.0f;
            const float *wr = W0 + (size_t)ti * NN * ND + v;
#pragma unroll 10
            for (int mu = 0; mu < NN; ++mu) {
                const float wv = wr[(size_t)mu * ND];
#pragma unroll
                for (int g = 0; g < G; ++g) e[g] += wv * tail[g * NN + mu];
            }
            const float sc = scale[v];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                sm.at[g].ab[v] = e[g] * sc;
                if (g < nb) a.dqt[(size_t)(bp0 + g) * ND + v] = sm.at[g].dqt[v];
            }
        }
        __syncwarp();

        // ---------------------------------------------------------------- dJ/dA (in place of dA)
#pragma unroll
        for (int jj = 0; jj < NLMO; ++jj) {
            const int lm = sl + jj * SW;
            if (lm < L3) {
                const int l = l_of_lm(lm);
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float *An = at.A + n * L3;
                    const float *dAn = at.dA + n * L3;
                    const int v3 = NR + (l - 1) * NA + n;
                    float x = 2.0f * at.ab[v3] * An[lm] + 2.0f * at.b[v3] * dAn[lm];
                    if (l == 2)
                        x += at.ab[NR + 4 * NA + n] * at.G4[n * 5 + lm - 3] + at.b[NR + 4 * NA + n] * at.H4[n * 5 + lm - 3];
                    if (l == 1) {
                        const float q1 = An[0] * An[0] + An[1] * An[1] + An[2] * An[2];
                        const int v5 = NR + 5 * NA + n;
                        x += at.ab[v5] * 4.0f * q1 * An[lm] + at.b[v5] * (8.0f * at.ad[n] * An[lm] + 4.0f * q1 * dAn[lm]);
                    }
                    at.dA[n * L3 + lm] = x;  // only this lane reads or writes element (n, lm) here
                }
            }
        }
        __syncwarp();

        // ---------------------------------------------------------------- radial coefficient gradient
#pragma unroll 1
        for (int g2 = 0; g2 < G; ++g2) {
            if (grp == g2) {
                for (int e = sl; e < T * NCR; e += SW) {
                    const int bb = e / NCR, rr = e - bb * NCR, n = rr / KR, kk = rr - n * KR;
                    accR[e] += at.ab[n] * Sr[bb * 2 * KR + kk] + at.b[n] * Sr[bb * 2 * KR + KR + kk];
                }
            }
            __syncwarp();
        }

        // ---------------------------------------------------------------- angular coefficient gradient
        {
            const float *Ab = at.dA;
            float X[VA];
#pragma unroll
            for (int e = 0; e < VA; ++e) X[e] = 0.0f;
            int bcur = -1;
            float4 nxt = pair_or_zero(prs, sl, nAng);
            for (int c0 = 0; c0 < maxA; c0 += SW) {
                const int k = c0 + sl;
                const bool valid = k < nAng;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nAng);
                int tj = -1;
                float f[KA], fp[KA], al[NA], be[NA];
#pragma unroll
                for (int kk = 0; kk < KA; ++kk) f[kk] = fp[kk] = 0.0f;
#pragma unroll
                for (int n = 0; n < NA; ++n) al[n] = be[n] = 0.0f;
                if (valid) {
                    const int j = pair_j(pd);
                    tj = pair_t(pd);
                    const float4 fbj = a.fbar[j];
                    const float lx = fbx - fbj.x - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
                    const float ly = fby - fbj.y - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
                    const float lz = fbz - fbj.z - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    const float r = r2 * rinv;
                    const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
                    const float rl = ux * lx + uy * ly + uz * lz;
                    const float px = (lx - rl * ux) * rinv, py = (ly - rl * uy) * rinv, pz = (lz - rl * uz) * rinv;
                    basis_val_der<KA>(r, a.inv_rcA, f, fp);
                    ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                        const float ps = gx * px + gy * py + gz * pz;
#pragma unroll
                        for (int n = 0; n < NA; ++n) {
                            const float ah = at.Ah[n * L3 + lm];
                            al[n] += Ab[n * L3 + lm] * Y + ah * ps;
                            be[n] += ah * Y;
                        }
                    });
#pragma unroll
                    for (int n = 0; n < NA; ++n) be[n] *= rl;
                }
                if (T == 1) {  // one species: no runs to track
                    if (valid) {
#pragma unroll
                        for (int n = 0; n < NA; ++n)
#pragma unroll
                            for (int kk = 0; kk < KA; ++kk) X[n * KA + kk] += al[n] * f[kk] + be[n] * fp[kk];
                    }
                    continue;
                }
                unsigned rem = group_bits<SW>(__ballot_sync(FULL, valid), lane);
                while (__any_sync(FULL, rem != 0)) {
                    const bool has = rem != 0;
                    const int leader = has ? __ffs(rem) - 1 : 0;
                    int bsp = __shfl_sync(FULL, tj, (lane & ~(SW - 1)) + leader);
                    if (!has) bsp = bcur;
                    const bool inb = valid && has && tj == bsp;
                    rem &= ~group_bits<SW>(__ballot_sync(FULL, inb), lane);
                    const bool change = bsp != bcur;
                    if (__any_sync(FULL, change && bcur >= 0))
                        flush_groups<VA, SW>(X, accA + (bcur >= 0 ? bcur : 0) * NCA, NCA, bcur >= 0, lane, true);
                    bcur = bsp;
                    if (inb) {
#pragma unroll
                        for (int n = 0; n < NA; ++n)
#pragma unroll
                            for (int kk = 0; kk < KA; ++kk) X[n * KA + kk] += al[n] * f[kk] + be[n] * fp[kk];
                    }
                }
            }
            if (T == 1 && nAng > 0) bcur = 0;
            if (__any_sync(FULL, bcur >= 0))
                flush_groups<VA, SW>(X, accA + (bcur >= 0 ? bcur : 0) * NCA, NCA, bcur >= 0, lane, true);
        }
        __syncwarp();
    }
    __syncwarp();
    if (cur_t >= 0) flush_slot(cur_t);
}

// ============================================================================= dispatch

template <class S, int SW, int VAR>
void launch_fwd_t(const AtomArgs &a, int blocks, int wpb, size_t smem, cudaStream_t st) {
    k_forward<S, SW, VAR><<<blocks, wpb * 32, smem, st>>>(a);
}
template <class S, int SW, int VAR>
void launch_adj_t(const AtomArgs &a, int blocks, int wpb, size_t smem, cudaStream_t st) {
    k_adjoint<S, SW, VAR><<<blocks, wpb * 32, smem, st>>>(a);
}
template <class S, int SW>
size_t fwd_bytes_t(int T, int NN) { return FwdL<S, SW>::bytes(T, NN); }
template <class S, int SW>
size_t adj_bytes_t(int T, int NN) { return AdjL<S, SW>::bytes(T, NN); }

// Variant v: SW = 8 (v < 2) or 16, register budget VAR = v & 1.
template <int NR, int KR, int NA, int KA>
KernelSet make_set() {
    using S = Shape<NR, KR, NA, KA>;
    KernelSet k;
    k.NR = NR;
    k.KR = KR;
    k.NA = NA;
    k.KA = KA;
    k.fwd_fn[0] = (const void *)k_forward<S, 8, 0>;
    k.fwd_fn[1] = (const void *)k_forward<S, 8, 1>;
    k.fwd_fn[2] = (const void *)k_forward<S, 16, 0>;
    k.fwd_fn[3] = (const void *)k_forward<S, 16, 1>;
    k.adj_fn[0] = (const void *)k_adjoint<S, 8, 0>;
    k.adj_fn[1] = (const void *)k_adjoint<S, 8, 1>;
    k.adj_fn[2] = (const void *)k_adjoint<S, 16, 0>;
    k.adj_fn[3] = (const void *)k_adjoint<S, 16, 1>;
    k.launch_fwd[0] = launch_fwd_t<S, 8, 0>;
    k.launch_fwd[1] = launch_fwd_t<S, 8, 1>;
    k.launch_fwd[2] = launch_fwd_t<S, 16, 0>;
    k.launch_fwd[3] = launch_fwd_t<S, 16, 1>;
    k.launch_adj[0] = launch_adj_t<S, 8, 0>;
    k.launch_adj[1] = launch_adj_t<S, 8, 1>;
    k.launch_adj[2] = launch_adj_t<S, 16, 0>;
    k.launch_adj[3] = launch_adj_t<S, 16, 1>;
    k.fwd_smem[0] = k.fwd_smem[1] = fwd_bytes_t<S, 8>;
    k.fwd_smem[2] = k.fwd_smem[3] = fwd_bytes_t<S, 16>;
    k.adj_smem[0] = k.adj_smem[1] = adj_bytes_t<S, 8>;
    k.adj_smem[2] = k.adj_smem[3] = adj_bytes_t<S, 16>;
    for (int v = 0; v < NVAR; ++v) {
        k.max_wpb[v] = (v & 1) ? 8 : 4;
        k.sw[v] = v < 2 ? 8 : 16;
    }
    return k;
}

}  // namespace nep
