// Parameter expansion, the force gather, per-structure sums and the E/F/W loss in one
// launch, the network-gradient contraction, and the deterministic reduction of the
// parameter gradient (with the optimiser step in training).
//
// Fixed-order reductions everywhere: sums in a fixed lane order, per-block partials in a
// fixed warp order, and a final pass over the partials in index order (compensated FP32
// pair sums where FP64 would serialise on this part's slow FP64 units).  No floating-point
// atomics, so two runs with the same launch shape are bit-identical.
#include <algorithm>
#include <vector>

#include "nep_ctx.cuh"


namespace nep {

namespace {

// --------------------------------------------------------------------------- parameters
struct ExpandArgs {
    const float *theta, *qscale;
    float *par;
    ParOff po;
    int T, NN, NDc, NDP, nR, kR, nA, kA, NRP, KRP, NAP, KAP;
    const int *inv;  // [NDP] padded -> compact descriptor index, -1 for padding
};

__global__ void k_expand(ExpandArgs x) {
    grid_dep_wait();
    grid_dep_launch();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ParOff &po = x.po;
    if (e >= po.total) return;
    const int T = x.T, NN = x.NN, ND = x.NDc, NDP = x.NDP;
    const int64_t cb0 = (int64_t)T * NN * ND, cw1 = cb0 + (int64_t)T * NN, cb1 = cw1 + (int64_t)T * NN;
    const int64_t ccR = cb1 + 1, ccA = ccR + (int64_t)T * T * x.nR * x.kR;
    float v = 0.0f;
    if (e < po.w0t) {
        const int64_t r = e - po.w0;
        const int vp = (int)(r % NDP);
        const int64_t tm = r / NDP;  // t*NN + mu
        const int vc = x.inv[vp];
        if (vc >= 0) v = x.theta[tm * ND + vc];
    } else if (e < po.b0) {
        const int64_t r = e - po.w0t;
        const int mu = (int)(r % NN);
        const int64_t tv = r / NN;  // t*NDP + vp
        const int vp = (int)(tv % NDP), t = (int)(tv / NDP);
        const int vc = x.inv[vp];
        if (vc >= 0) v = x.theta[((int64_t)t * NN + mu) * ND + vc];
    } else if (e < po.w1) {
        v = x.theta[cb0 + (e - po.b0)];
    } else if (e < po.b1) {
        v = x.theta[cw1 + (e - po.w1)];
    } else if (e < po.cR) {
        v = (e == po.b1) ? x.theta[cb1] : 0.0f;
    } else if (e < po.cA) {
        const int64_t r = e - po.cR;
        const int k = (int)(r % x.KRP);
        const int n = (int)((r / x.KRP) % x.NRP);
        const int64_t ab = r / ((int64_t)x.KRP * x.NRP);
        if (n < x.nR && k < x.kR) v = x.theta[ccR + (ab * x.nR + n) * x.kR + k];
    } else if (e < po.scale) {
        const int64_t r = e - po.cA;
        const int k = (int)(r % x.KAP);
        const int n = (int)((r / x.KAP) % x.NAP);
        const int64_t ab = r / ((int64_t)x.KAP * x.NAP);
        if (n < x.nA && k < x.kA) v = x.theta[ccA + (ab * x.nA + n) * x.kA + k];
    } else if (e < po.cRp) {
        const int64_t r = e - po.scale;
        const int vc = r < NDP ? x.inv[r] : -1;
        if (vc >= 0) v = x.qscale[vc];
    } else if (e < po.cAp) {
        const int K4 = round4(x.KRP);
        const int64_t r = e - po.cRp;
        const int k = (int)(r % K4);
        const int n = (int)((r / K4) % x.NRP);
        const int64_t ab = r / ((int64_t)K4 * x.NRP);
        if (n < x.nR && k < x.kR) v = x.theta[ccR + (ab * x.nR + n) * x.kR + k];
    } else {
        const int K4 = round4(x.KAP);
        const int64_t r = e - po.cAp;
        const int k = (int)(r % K4);
        const int n = (int)((r / K4) % x.NAP);
        const int64_t ab = r / ((int64_t)K4 * x.NAP);
        if (n < x.nA && k < x.kA) v = x.theta[ccA + (ab * x.nA + n) * x.kA + k];
    }
    x.par[e] = v;
}

// --------------------------------------------------------------------------- loss terms
struct TermsArgs {
    int64_t a0, a1, s0, s1;
    int nG;  // the first nG blocks gather forces, the next s1 - s0 sum one structure each
    const int64_t *nbr_off;
    const int *rev;
    const float4 *G;
    const float *F_own;
    float *F_out;
    const int64_t *atom_off;
    const float *E_atom, *W_atom;
    double *E_out, *W_out;
    int loss;
    const float *F_ref;
    float coefF;
    float *fbar;
    const double *E_ref, *W_ref;
    const uint8_t *has_W;
    const int *n_sv;  // device count of N_s^V when nsv <= 0
    double nsv, lamE, lamV, Ns, Na;
    float *ebar, *wbar;
    double *fpart, *spart;  // [nG] force partials; [3 (s1 - s0)] structure partials
    double *loss3, *gb1;    // loss3: the last block reduces the partials
    unsigned *counter;
};

// F_i = sum_{p in N(i)} G_p - sum_{p in N(i)} G_{rev(p)}: the second sum visits the pairs
// (j, i, -S) of which i is the neighbour, through the reverse index (no atomics).  Each
// half-warp takes one atom (two atoms in flight per warp) and the half-warps stride over the
// atoms; the next atom's list bounds are loaded while the current atom's rows are gathered.
// The block's squared force residuals go to fpart[block].
__device__ void gather_block(const TermsArgs &x, int blk) {
    __shared__ float2 wpart[32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int hl = lane & 15;
    const int64_t H = (int64_t)x.nG * nw * 2;
    int64_t i = x.a0 + ((int64_t)blk * nw + wib) * 2 + (lane >> 4);
    int64_t beg = 0, end = 0;
    if (i < x.a1) {
        beg = x.nbr_off[i];
        end = x.nbr_off[i + 1];
    }
    float ah = 0.0f, al = 0.0f;  // sum of d^2: each square exact as p + e (FMA), then TwoSum
    while (__any_sync(FULL, i < x.a1)) {
        const int64_t in = i + H;
        int64_t nbeg = 0, nend = 0;
        if (in < x.a1) {
            nbeg = x.nbr_off[in];
            nend = x.nbr_off[in + 1];
        }
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for (int64_t p0 = beg; p0 < end; p0 += 128) {  // 8 index loads, then 8 gathers, in flight
            int r[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t p = p0 + hl + 16 * k;
                r[k] = p < end ? x.rev[p] : -1;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (r[k] >= 0) {
                    const float4 g = x.G[r[k]];
                    sx += g.x;
                    sy += g.y;
                    sz += g.z;
                }
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {  // sums over each half-warp
            sx += __shfl_xor_sync(FULL, sx, o);
            sy += __shfl_xor_sync(FULL, sy, o);
            sz += __shfl_xor_sync(FULL, sz, o);
        }
        if (hl < 3 && i < x.a1) {
            const float own = x.F_own[i * 3 + hl];
            const float F = own - (hl == 0 ? sx : hl == 1 ? sy : sz);
            x.F_out[i * 3 + hl] = F;
            if (x.loss) {
                const float d = F - x.F_ref[i * 3 + hl];
                x.fbar[i * 4 + hl] = x.coefF * d;  // float4 rows (x, y, z, unused)
                const float p = d * d;
                f2_add(ah, al, p);
                al += fmaf(d, d, -p);
            }
        }
        i = in;
        beg = nbeg;
        end = nend;
    }
    if (!x.loss) return;
    // lanes 0..2 and 16..18 hold the sums (the others zero): lanes 0 and 16 take their
    // half's 1 and 2, then lane 0 takes lane 16, in a fixed order
    f2_merge(ah, al, __shfl_down_sync(FULL, ah, 1), __shfl_down_sync(FULL, al, 1));
    f2_merge(ah, al, __shfl_down_sync(FULL, ah, 2), __shfl_down_sync(FULL, al, 2));
    f2_merge(ah, al, __shfl_down_sync(FULL, ah, 16), __shfl_down_sync(FULL, al, 16));
    if (lane == 0) wpart[wib] = make_float2(ah, al);
    __syncthreads();
    if (threadIdx.x == 0) {
        float h = 0.0f, l = 0.0f;
        for (int k = 0; k < nw; ++k) f2_merge(h, l, wpart[k].x, wpart[k].y);
        x.fpart[blk] = (double)h + (double)l;
    }
}

// E_s = sum_i E_i and W_s = sum_i W_i (Eq. 1) as compensated FP32 pair sums, returned in
// FP64; loss terms and cotangents of Eq. "loss".  The block's threads stride over the
// structure's atoms, then a fixed-order reduction (lanes, then warps in order), so a
// 10,000-atom cell is summed by all 256 threads.  Lanes k = 0..9 of warp 0 finish one
// quantity each (0: E, 1..9: W).  spart[3 (s - s0) + q]: the structure's loss terms.
__device__ void struct_block(const TermsArgs &x, int64_t s) {
    __shared__ float2 red[10][33];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b = x.atom_off[s], e = x.atom_off[s + 1];
    float h[10], l[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) h[k] = l[k] = 0.0f;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        f2_add(h[0], l[0], x.E_atom[i]);
#pragma unroll
        for (int k = 0; k < 9; ++k) f2_add(h[1 + k], l[1 + k], x.W_atom[i * 9 + k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 10; ++k)
            f2_merge(h[k], l[k], __shfl_xor_sync(FULL, h[k], o), __shfl_xor_sync(FULL, l[k], o));
    if (lane < 10) {
#pragma unroll
        for (int k = 0; k < 10; ++k)
            if (k == lane) red[k][wib] = make_float2(h[k], l[k]);
    }
    __syncthreads();
    if (wib != 0) return;
    double v = 0.0;  // lane k: the finished quantity k
    if (lane < 10) {
        float hh = 0.0f, ll = 0.0f;
        for (int w = 0; w < nw; ++w) f2_merge(hh, ll, red[lane][w].x, red[lane][w].y);
        v = (double)hh + (double)ll;
        if (lane == 0) x.E_out[s] = v;
        else x.W_out[s * 9 + lane - 1] = v;
    }
    if (!x.loss) return;
    // FP64 division is slow on this part: one reciprocal per lane, coefficients once
    const double NsV = x.nsv > 0.0 ? x.nsv : (double)(*x.n_sv);
    const double na = (double)(e - b);
    const double inv_na = 1.0 / na, inv_na2 = inv_na * inv_na;
    const bool hw = x.has_W == nullptr || x.has_W[s] != 0;
    double aV = 0.0;
    if (lane >= 1 && lane < 10) {
        double wb = 0.0;
        if (hw && NsV > 0.0) {
            const double dW = v - x.W_ref[s * 9 + lane - 1];
            aV = (dW * inv_na) * (dW * inv_na);
            wb = (x.lamV * 2.0 / (9.0 * NsV)) * dW * inv_na2;
        }
        x.wbar[s * 9 + lane - 1] = (float)wb;
    }
    // lanes 1..9 in order onto lane 0 (fixed order)
    double tV = 0.0;
    for (int k = 1; k < 10; ++k) tV += __shfl_sync(FULL, aV, k);
    if (lane == 0) {
        const double dE = v - x.E_ref[s];
        const double eb = (x.lamE * 2.0 / x.Ns) * dE * inv_na2;
        x.ebar[s] = (float)eb;
        x.spart[3 * (s - x.s0) + 0] = (dE * inv_na) * (dE * inv_na);
        x.spart[3 * (s - x.s0) + 1] = tV;
        x.spart[3 * (s - x.s0) + 2] = -na * eb;
    }
}

// The loss terms DeltaE, DeltaF, DeltaV of Eq. "loss" and dL/db1 from the partials, in a
// fixed order (strided thread sums, lanes, then warps in order).  Partials written by
// other blocks of the same launch are read through L2.
__device__ void loss_reduce(const double *fpart, int nf, const double *spart, int nsb, double nsv, double Ns,
                            double Na, double *loss3, double *gb1) {
    __shared__ double sh[32][4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nsb; k += blockDim.x) {
        a[0] += __ldcg(spart + 3 * k);
        a[2] += __ldcg(spart + 3 * k + 1);
        a[3] += __ldcg(spart + 3 * k + 2);
    }
    for (int k = threadIdx.x; k < nf; k += blockDim.x) a[1] += __ldcg(fpart + k);
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = warp_sum_d(a[q]);
    if (lane == 0)
        for (int q = 0; q < 4; ++q) sh[wib][q] = a[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < nw; ++w)
            for (int q = 0; q < 4; ++q) t[q] += sh[w][q];
        loss3[0] = Ns > 0 ? t[0] / Ns : 0.0;
        loss3[1] = Na > 0 ? t[1] / (3.0 * Na) : 0.0;
        loss3[2] = nsv > 0 ? t[2] / (9.0 * nsv) : 0.0;
        *gb1 = t[3];
    }
}

// Force gather, structure sums and (with loss3) the loss reduction in one launch of
// 256-thread blocks: the reduction runs in the block that finishes last.
__global__ void __launch_bounds__(256) k_loss_terms(TermsArgs x) {
    grid_dep_wait();
    grid_dep_launch();
    const int blk = blockIdx.x;
    if (blk < x.nG) gather_block(x, blk);
    else struct_block(x, x.s0 + (blk - x.nG));
    if (!x.loss || !x.loss3) return;
    if (!last_block_arrival(x.counter, gridDim.x, threadIdx.x == 0)) return;
    const double nsv = x.nsv > 0.0 ? x.nsv : (double)__ldcg(x.n_sv);
    loss_reduce(x.fpart, x.nG, x.spart, (int)(x.s1 - x.s0), nsv, x.Ns, x.Na, x.loss3, x.gb1);
}

__global__ void k_count_hasw(int64_t ns, const uint8_t *has_W, int *n_sv) {
    grid_dep_wait();
    grid_dep_launch();
    __shared__ int sh[256];
    int c = 0;
    for (int64_t s = threadIdx.x; s < ns; s += blockDim.x) c += (has_W == nullptr || has_W[s]) ? 1 : 0;
    sh[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) t += sh[k];
        *n_sv = t;
    }
}

// Loss reduction over partials left by several launches (plain form).
__global__ void k_loss_final(const double *fpart, int nf, const double *spart, int nsb, const int *n_sv,
                             double nsv, double Ns, double Na, double *loss3, double *gb1) {
    const double v = nsv > 0.0 ? nsv : (double)(*n_sv);
    loss_reduce(fpart, nf, spart, nsb, v, Ns, Na, loss3, gb1);
}

// dL/dF rows into the float4 layout the adjoint gathers.
__global__ void k_fbar_rows(int64_t na, const float *dF, float4 *fbar) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < na) fbar[i] = make_float4(dF[3 * i], dF[3 * i + 1], dF[3 * i + 2], 0.0f);
}

// Cotangents supplied by the caller (vector-Jacobian product for autograd).
__global__ void k_cotangents(int64_t ns, const int64_t *atom_off, const double *dE, const double *dW, float *ebar,
                             float *wbar, double *gb1) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int64_t s = threadIdx.x; s < ns; s += blockDim.x) {
        ebar[s] = (float)dE[s];
        for (int k = 0; k < 9; ++k) wbar[s * 9 + k] = (float)dW[s * 9 + k];
        a -= (double)(atom_off[s + 1] - atom_off[s]) * dE[s];
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *gb1 = sh[0];
}

// --------------------------------------------------------------------------- network gradient
// grad_w0[t] = sum_i zeta_i q~_i^T + u_i dq~_i^T, grad_b0[t] = -sum zeta, grad_w1[t] = sum omega
// over the atoms of species t: a contraction over atoms ([NN x 2n] . [2n x ND]).  One
// block per chunk of work positions holding a single species (more only when the 4 x 4
// tiles of the NN x ND output outnumber 256 threads); each thread accumulates one 4 x 4
// register tile; FP32 partial per chunk.
constexpr int ANN_ROWS = 32;
constexpr int ANN_MAX_THREADS = 256;

// Asynchronous 4-byte global -> shared copy (zero fill when !pred), so that the next rows
// of a chunk load while the current ones are contracted.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct AnnTile {  // one buffer of ANN_ROWS staged rows
    float *z, *u, *o, *q, *d;
};

__device__ __forceinline__ AnnTile ann_tile(float *base, int NNP, int NDQ) {
    AnnTile t;
    t.z = base;
    t.u = t.z + ANN_ROWS * NNP;
    t.o = t.u + ANN_ROWS * NNP;
    t.q = t.o + ANN_ROWS * NNP;
    t.d = t.q + ANN_ROWS * NDQ;
    return t;
}

__device__ __forceinline__ void ann_stage(const AnnTile &t, int rr, int nr, int NN, int NDP, int NNP, int NDQ,
                                          const float *zt, const float *ut, const float *om, const float *qt,
                                          const float *dqt) {
    for (int e = threadIdx.x; e < ANN_ROWS * NNP; e += blockDim.x) {
        const int r = e / NNP, m = e - r * NNP;
        const bool in = r < nr && m < NN;
        const size_t g = in ? (size_t)(rr + r) * NN + m : 0;
        cp_async4(t.z + e, zt + g, in);
        cp_async4(t.u + e, ut + g, in);
        cp_async4(t.o + e, om + g, in);
    }
    for (int e = threadIdx.x; e < ANN_ROWS * NDQ; e += blockDim.x) {
        const int r = e / NDQ, v = e - r * NDQ;
        const bool in = r < nr && v < NDP;
        const size_t g = in ? (size_t)(rr + r) * NDP + v : 0;
        cp_async4(t.q + e, qt + g, in);
        cp_async4(t.d + e, dqt + g, in);
    }
    cp_async_commit();
}

__global__ void k_ann_grad(const int *chunk_begin, int NN, int NDP, const float *zt, const float *ut,
                           const float *om, const float *qt, const float *dqt, float *part) {
    grid_dep_wait();
    grid_dep_launch();
    extern __shared__ __align__(16) float sm[];
    const int NNP = (NN + 3) & ~3, NDQ = (NDP + 3) & ~3;
    const int tile_floats = ANN_ROWS * (3 * NNP + 2 * NDQ);
    const AnnTile buf[2] = {ann_tile(sm, NNP, NDQ), ann_tile(sm + tile_floats, NNP, NDQ)};
    const int c = blockIdx.x;
    const int r0 = chunk_begin[c], r1 = chunk_begin[c + 1];
    const int tn = NDQ / 4, ntiles = (NNP / 4) * tn;
    const int tile = blockIdx.y * blockDim.x + threadIdx.x;
    const bool own = tile < ntiles;
    const int mu0 = own ? 4 * (tile / tn) : 0, v0 = own ? 4 * (tile % tn) : 0;
    const bool first = blockIdx.y == 0;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
    float azeta = 0.0f, aom = 0.0f;
    if (r0 < r1) ann_stage(buf[0], r0, min(ANN_ROWS, r1 - r0), NN, NDP, NNP, NDQ, zt, ut, om, qt, dqt);
    int cur = 0;
    for (int rr = r0; rr < r1; rr += ANN_ROWS) {
        const int nr = min(ANN_ROWS, r1 - rr);
        cp_async_wait_all();
        __syncthreads();  // rows rr.. are in buf[cur]; every thread is done with buf[cur ^ 1]
        if (rr + ANN_ROWS < r1)
            ann_stage(buf[cur ^ 1], rr + ANN_ROWS, min(ANN_ROWS, r1 - rr - ANN_ROWS), NN, NDP, NNP, NDQ, zt, ut, om,
                      qt, dqt);
        const AnnTile &t = buf[cur];
        if (own) {
            for (int r = 0; r < nr; ++r) {
                const float4 z4 = *reinterpret_cast<const float4 *>(t.z + r * NNP + mu0);
                const float4 u4 = *reinterpret_cast<const float4 *>(t.u + r * NNP + mu0);
                const float4 q4 = *reinterpret_cast<const float4 *>(t.q + r * NDQ + v0);
                const float4 d4 = *reinterpret_cast<const float4 *>(t.d + r * NDQ + v0);
                const float z[4] = {z4.x, z4.y, z4.z, z4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w};
                const float q[4] = {q4.x, q4.y, q4.z, q4.w}, d[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] += z[x] * q[y] + uu[x] * d[y];
            }
        }
        if (first && (int)threadIdx.x < NN) {
            for (int r = 0; r < nr; ++r) {
                azeta += t.z[r * NNP + threadIdx.x];
                aom += t.o[r * NNP + threadIdx.x];
            }
        }
        cur ^= 1;
    }
    const int nent = NN * NDP;
    float *dst = part + (size_t)c * (nent + 2 * NN);
    if (own) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y)
                if (mu0 + x < NN && v0 + y < NDP) dst[(mu0 + x) * NDP + v0 + y] = acc[x][y];
    }
    if (first && (int)threadIdx.x < NN) {
        dst[nent + threadIdx.x] = azeta;
        dst[nent + NN + threadIdx.x] = aom;
    }
}

// --------------------------------------------------------------------------- final gradient
struct GradArgs {
    int T, NN, ND, NDP, nR, kR, nA, kA, NRP, KRP, NAP, KAP;
    int64_t P;
    const int *desc_map;  // compact -> padded
    const float *annpart;
    const int *clo, *chi;  // [T] chunk range of each species
    const float *cpart;
    const int *wlo, *whi;  // [T] adjoint warp range of each species
    const int *warp_begin; // [W+1] adjoint schedule (warps without atoms wrote no slot)
    const double *gb1;
    float *grad;
    double *acc;           // plain form: add the partial sums here (FP64), b1 left out
    unsigned *counters;    // [0] all columns done, [1 + x] segments of column x done
    int opt;               // training: AMSGrad step on each parameter once its gradient is final
    OptArgs o;
};

// One launch, one block per (32 consecutive parameters = a column, row segment), with
// GF_RG row groups (threadIdx.y): the threads of a warp read 32 neighbouring parameters of
// one partial row (coalesced), each thread keeps two compensated FP32 pair sums, the row
// groups are merged pairwise in a fixed order and each segment's sum goes to gpart[seg][k].
// The last of a column's GF_SEG blocks to finish merges the segments in order (the final
// gradient), and in training applies the optimiser step to those parameters; the last
// column then advances the optimiser state.  Spreading the rows over segments keeps every
// SM busy.
constexpr int GF_RG = 16;
constexpr int GF_SEG = 8;

struct GradSource {  // where parameter k's partials live
    bool net;         // network parameter: rows = chunks [lo, hi) of annpart
    bool b1;          // the shared output bias (from the loss reduction)
    int lo, hi;       // row range (c-parameters: adjoint warps [lo, hi), slot w + a)
    int a, b, off;    // species pair of a c-parameter, column in the partial row
    double sign;
};

__device__ __forceinline__ GradSource grad_source(const GradArgs &g, int64_t k) {
    GradSource r{};
    r.sign = 1.0;
    const int T = g.T, NN = g.NN, ND = g.ND;
    const int64_t cb0 = (int64_t)T * NN * ND, cw1 = cb0 + (int64_t)T * NN, cb1 = cw1 + (int64_t)T * NN;
    const int64_t ccR = cb1 + 1, ccA = ccR + (int64_t)T * T * g.nR * g.kR;
    const int NCR = g.NRP * g.KRP;
    if (k < cb1) {
        int t;
        r.net = true;
        if (k < cb0) {
            t = (int)(k / ((int64_t)NN * ND));
            const int rr = (int)(k - (int64_t)t * NN * ND);
            const int mu = rr / ND, v = rr - mu * ND;
            r.off = mu * g.NDP + g.desc_map[v];
        } else if (k < cw1) {
            t = (int)((k - cb0) / NN);
            r.off = NN * g.NDP + (int)((k - cb0) % NN);
            r.sign = -1.0;
        } else {
            t = (int)((k - cw1) / NN);
            r.off = NN * g.NDP + NN + (int)((k - cw1) % NN);
        }
        r.lo = g.clo[t];
        r.hi = g.chi[t];
    } else if (k == cb1) {
        r.b1 = true;
    } else {
        int64_t rr;
        int kk, n;
        if (k < ccA) {
            rr = k - ccR;
            kk = (int)(rr % g.kR);
            n = (int)((rr / g.kR) % g.nR);
            rr /= (int64_t)g.kR * g.nR;
            r.off = n * g.KRP + kk;
        } else {
            rr = k - ccA;
            kk = (int)(rr % g.kA);
            n = (int)((rr / g.kA) % g.nA);
            rr /= (int64_t)g.kA * g.nA;
            r.off = NCR + n * g.KAP + kk;
        }
        r.a = (int)(rr / T);
        r.b = (int)(rr % T);
        r.lo = g.wlo[r.a];
        r.hi = g.whi[r.a] + 1;
    }
    return r;
}

__global__ void __launch_bounds__(32 * GF_RG) k_grad_reduce(GradArgs g, float2 *gpart /*[GF_SEG][P]*/) {
    grid_dep_wait();
    grid_dep_launch();
    __shared__ float2 red[GF_RG][33];
    const int tx = threadIdx.x, ty = threadIdx.y, seg = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * 32 + tx;
    const int T = g.T, NC = g.NRP * g.KRP + g.NAP * g.KAP;
    const int annstride = g.NN * g.NDP + 2 * g.NN;
    float h = 0.0f, l = 0.0f;
    GradSource r{};
    if (k < g.P) {
        r = grad_source(g, k);
        if (!r.b1) {
            const int len = (r.hi - r.lo + GF_SEG - 1) / GF_SEG;
            const int lo = r.lo + seg * len, hi = min(r.hi, lo + len);
            // two compensated chains keep two loads in flight, merged in a fixed order
            float h2 = 0.0f, l2 = 0.0f;
            if (r.net) {
                int c = lo + ty;
                for (; c + GF_RG < hi; c += 2 * GF_RG) {
                    f2_add(h, l, g.annpart[(size_t)c * annstride + r.off]);
                    f2_add(h2, l2, g.annpart[(size_t)(c + GF_RG) * annstride + r.off]);
                }
                if (c < hi) f2_add(h, l, g.annpart[(size_t)c * annstride + r.off]);
            } else {
                int w = lo + ty;
                for (; w + GF_RG < hi; w += 2 * GF_RG) {
                    if (g.warp_begin[w] < g.warp_begin[w + 1])
                        f2_add(h, l, g.cpart[((size_t)(w + r.a) * T + r.b) * NC + r.off]);
                    const int w2 = w + GF_RG;
                    if (g.warp_begin[w2] < g.warp_begin[w2 + 1])
                        f2_add(h2, l2, g.cpart[((size_t)(w2 + r.a) * T + r.b) * NC + r.off]);
                }
                if (w < hi && g.warp_begin[w] < g.warp_begin[w + 1])
                    f2_add(h, l, g.cpart[((size_t)(w + r.a) * T + r.b) * NC + r.off]);
            }
            f2_merge(h, l, h2, l2);
        }
    }
    red[ty][tx] = make_float2(h, l);
    __syncthreads();
#pragma unroll
    for (int o = GF_RG / 2; o > 0; o >>= 1) {  // row groups pairwise, fixed pairing
        if (ty < o) {
            float2 a = red[ty][tx];
            const float2 b = red[ty + o][tx];
            f2_merge(a.x, a.y, b.x, b.y);
            red[ty][tx] = a;
        }
        __syncthreads();
    }
    const bool writer = ty == 0 && k < g.P;
    if (writer) gpart[(size_t)seg * g.P + k] = red[0][tx];
    if (!last_block_arrival(g.counters + 1 + blockIdx.x, GF_SEG, writer)) return;
    OptStep os{};
    if (g.opt) os = opt_step_state(g.o);
    if (writer) {
        float th = 0.0f, tl = 0.0f;
        for (int sg = 0; sg < GF_SEG; ++sg) {
            const float2 v = __ldcg(gpart + (size_t)sg * g.P + k);
            f2_merge(th, tl, v.x, v.y);
        }
        if (g.acc) {
            if (!r.b1) g.acc[k] += r.sign * ((double)th + (double)tl);
        } else {
            const float gk = r.b1 ? (float)*g.gb1 : (float)r.sign * (th + tl);
            g.grad[k] = gk;
            if (g.opt) amsgrad_elem(g.o, os, k, (double)gk);
        }
    }
    if (!g.opt) return;
    if (!last_block_arrival(g.counters, gridDim.x, false)) return;
    if (tx == 0 && ty == 0) opt_tick(g.o);
}

// Plain form: gradient = FP64 accumulator, b1 from the loss reduction.
__global__ void k_grad_convert(int64_t P, int64_t kb1, const double *acc, const double *gb1, float *grad) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) grad[k] = (float)(k == kb1 ? *gb1 : acc[k]);
}

// --------------------------------------------------------------------------- descriptor range
__global__ void k_range(int64_t na, int NDP, int ND, const int *desc_map, const float *q, float *qmin, float *qmax) {
    __shared__ float smin[256], smax[256];
    const int v = blockIdx.x;
    const int vp = desc_map[v];
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = threadIdx.x; i < na; i += blockDim.x) {
        const float x = q[i * NDP + vp];
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        qmin[v] = na > 0 ? smin[0] : 0.0f;
        qmax[v] = na > 0 ? smax[0] : 0.0f;
    }
}

__global__ void k_compact_q(int64_t na, int NDP, int ND, const int *desc_map, const float *qp, float *q) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= na * ND) return;
    const int64_t i = e / ND;
    const int v = (int)(e - i * ND);
    q[e] = qp[i * NDP + desc_map[v]];
}

}  // namespace

// =========================================================================== launchers

static AtomArgs atom_args(Ctx *c) {
    AtomArgs a{};
    a.work = c->work.as<int>();
    a.rec = c->rec.as<int4>();
    a.rec2 = c->rec2.as<int2>();
    a.nbr_off = c->nbr_off.as<int64_t>();
    a.n_ang = c->n_ang.as<int>();
    a.pair = (const float4 *)c->pair.ptr;
    a.type = c->type.as<int>();
    a.struct_of = c->struct_of.as<int>();
    a.par = c->par.as<float>();
    a.T = c->T;
    a.NN = c->NN;
    a.inv_rcR = 1.0f / c->cfg.rc_R;
    a.inv_rcA = 1.0f / c->cfg.rc_A;
    a.rc2A = c->cfg.rc_A * c->cfg.rc_A;
    a.zbl = c->zbl_r2 > 0.0f ? c->zbl_tab.as<float>() : nullptr;
    a.zbl_r1 = c->zbl_r1;
    a.zbl_r2 = c->zbl_r2;
    a.E_atom = c->E_atom.as<float>();
    a.F_own = c->F_own.as<float>();
    a.W_atom = c->W_atom.as<float>();
    a.G = (float4 *)c->G.ptr;
    a.st_qt = c->st_qt.as<float>();
    a.st_h = c->st_h.as<float>();
    a.st_A = c->st_A.as<float>();
    a.fbar = c->fbar.as<float4>();
    a.ebar = c->ebar.as<float>();
    a.wbar = c->wbar.as<float>();
    a.zt = c->zt.as<float>();
    a.ut = c->ut.as<float>();
    a.om = c->om.as<float>();
    a.dqt = c->dqt.as<float>();
    a.cpart = c->cpart.as<float>();
    a.chunks = c->chunk_begin.as<int>();
    a.n_chunks = c->n_chunks;
    a.chunk_rows = NET_CHUNK;  // the batch's chunks (nep_set_structures)
    a.NDP = c->NDP;
    a.st_D = c->st_D.as<float>();
    a.st_S = c->st_S.as<float>();
    a.st_b = c->st_b.as<float>();
    a.st_ab = c->st_ab.as<float>();
    a.st_E = c->st_E.as<float>();
    return a;
}

namespace {
__global__ void k_work_rec(int64_t n, const int *work, const int *type, const int *struct_of, const int64_t *nbr_off,
                           const int *n_ang, int4 *rec, int2 *rec2) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = work[q];
    const int64_t b = nbr_off[i];
    rec[q] = make_int4(i, (int)b, (int)(nbr_off[i + 1] - b), n_ang[i]);
    rec2[q] = make_int2(type[i], struct_of[i]);
}
}  // namespace

int build_work_rec(Ctx *c, const int *work, DevBuf &rec, DevBuf &rec2) {
    const int64_t na = c->n_atoms;
    if (rec.ensure<int4>(na) || rec2.ensure<int2>(na)) return c->fail(NEP_ENOMEM, "work records");
    if (na == 0) return NEP_OK;
    k_work_rec<<<(unsigned)((na + 255) / 256), 256, 0, c->stream>>>(na, work, c->type.as<int>(), c->struct_of.as<int>(),
                                                                    c->nbr_off.as<int64_t>(), c->n_ang.as<int>(),
                                                                    rec.as<int4>(), rec2.as<int2>());
    CK_LAUNCH("k_work_rec");
    return NEP_OK;
}

int launch_expand(Ctx *c) {
    ExpandArgs x;
    x.theta = c->theta.as<float>();
    x.qscale = c->qscale.as<float>();
    x.par = c->par.as<float>();
    x.po = c->po;
    x.T = c->T;
    x.NN = c->NN;
    x.NDc = c->ND;
    x.NDP = c->NDP;
    x.nR = c->nR;
    x.kR = c->kR;
    x.nA = c->nA;
    x.kA = c->kA;
    x.NRP = c->ks->NR;
    x.KRP = c->ks->KR;
    x.NAP = c->ks->NA;
    x.KAP = c->ks->KA;
    x.inv = c->d_desc_inv.as<int>();
    const int64_t n = c->po.total;
    CK(launch_k(c->pdl(), k_expand, (unsigned)((n + 255) / 256), 256, 0, c->stream, x));
    return NEP_OK;
}

int launch_forward(Ctx *c, float *q_raw, int stage) {
    if (c->n_atoms == 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.warp_begin = c->fwd.warp_begin.as<int>();
    a.q_raw = q_raw;
    c->ks->launch_fwd[c->fwd.var](a, c->fwd.blocks, c->fwd.wpb, stage, c->stream, c->pdl());
    CK_LAUNCH("forward stages");
    return NEP_OK;
}

int launch_adjoint(Ctx *c, int stage) {
    if (c->n_atoms == 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.warp_begin = c->adj.warp_begin.as<int>();
    c->ks->launch_adj[c->adj.var](a, c->adj.blocks, c->adj.wpb, stage, c->stream, c->pdl());
    CK_LAUNCH("adjoint stages");
    return NEP_OK;
}

int launch_forward_sched(Ctx *c, const int *work, const DevBuf &rec, const DevBuf &rec2, const int *warp_begin,
                         int blocks, int var, int wpb, const int *chunks, int n_chunks, int chunk_rows) {
    if (blocks <= 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.work = work;
    a.rec = rec.as<int4>();
    a.rec2 = rec2.as<int2>();
    a.warp_begin = warp_begin;
    a.chunks = chunks;
    a.n_chunks = n_chunks;
    a.chunk_rows = chunk_rows;
    c->ks->launch_fwd[var](a, blocks, wpb, -1, c->stream, c->pdl());
    CK_LAUNCH("forward stages");
    return NEP_OK;
}

int launch_adjoint_sched(Ctx *c, const int *work, const DevBuf &rec, const DevBuf &rec2, const int *warp_begin,
                         int blocks, int var, int wpb, const int *chunks, int n_chunks, int chunk_rows) {
    if (blocks <= 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.work = work;
    a.rec = rec.as<int4>();
    a.rec2 = rec2.as<int2>();
    a.warp_begin = warp_begin;
    a.chunks = chunks;
    a.n_chunks = n_chunks;
    a.chunk_rows = chunk_rows;
    c->ks->launch_adj[var](a, blocks, wpb, -1, c->stream, c->pdl());
    CK_LAUNCH("adjoint stages");
    return NEP_OK;
}

// 8-warp gather blocks (two atoms in flight per warp): four per SM, and one block per 8 atoms
// for batches too small to fill them
static int gather_blocks(Ctx *c, int64_t n_atoms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(c->n_sm * 4, (n_atoms + 7) / 8));
}


double host_nsv(Ctx *c, const uint8_t *has_W, int64_t s0, int64_t s1) {
    int64_t n;
    if (!has_W) n = s1 - s0;
    else if (has_W == c->tgt_hw.as<uint8_t>() && c->tgt_has_hw && (int64_t)c->tgt_nsv_pre.size() > s1)
        n = c->tgt_nsv_pre[s1] - c->tgt_nsv_pre[s0];
    else return 0.0;
    return n > 0 ? (double)n : 1.0;
}

int launch_count_hasw(Ctx *c, const uint8_t *has_W, int64_t s0, int64_t s1) {
    CK(launch_k(c->pdl(), k_count_hasw, 1, 256, 0, c->stream, s1 - s0, has_W ? has_W + s0 : nullptr,
                c->n_sv.as<int>()));
    return NEP_OK;
}

int launch_terms(Ctx *c, const TermsCall &t) {
    const int64_t ns = t.s1 - t.s0;
    const int nG = t.a1 > t.a0 ? (t.gather_blocks > 0 ? t.gather_blocks : gather_blocks(c, t.a1 - t.a0)) : 0;
    if (nG + ns == 0)  // nothing to sum: the loss terms and dL/db1 are zero
        return t.loss && t.loss3 ? launch_loss_final(c, t.loss3, nullptr, 0, nullptr, 0, 1.0) : NEP_OK;
    TermsArgs x{};
    x.a0 = t.a0;
    x.a1 = t.a1;
    x.s0 = t.s0;
    x.s1 = t.s1;
    x.nG = nG;
    x.nbr_off = c->nbr_off.as<int64_t>();
    x.rev = c->rev.as<int>();
    x.G = (const float4 *)c->G.ptr;
    x.F_own = c->F_own.as<float>();
    x.F_out = t.F_out;
    x.atom_off = c->atom_off.as<int64_t>();
    x.E_atom = c->E_atom.as<float>();
    x.W_atom = c->W_atom.as<float>();
    x.E_out = t.E_out;
    x.W_out = t.W_out;
    x.loss = t.loss ? 1 : 0;
    x.F_ref = t.F_ref;
    x.coefF = (float)(t.lF * 2.0 / (3.0 * c->norm_Na()));
    x.fbar = c->fbar.as<float>();
    x.E_ref = t.E_ref;
    x.W_ref = t.W_ref;
    x.has_W = t.has_W;
    x.n_sv = c->n_sv.as<int>();
    x.nsv = t.nsv;
    x.lamE = t.lE;
    x.lamV = t.lV;
    x.Ns = c->norm_Ns();
    x.Na = c->norm_Na();
    x.ebar = c->ebar.as<float>();
    x.wbar = c->wbar.as<float>();
    x.fpart = t.fpart ? t.fpart : c->loss_part.as<double>();
    x.spart = t.spart ? t.spart : x.fpart + nG;
    x.loss3 = t.loss ? t.loss3 : nullptr;
    x.gb1 = c->gb1.as<double>();
    x.counter = c->counters.as<unsigned>();
    if (t.loss && t.nsv == 0.0) {
        if (int rc = launch_count_hasw(c, t.has_W, t.s0, t.s1)) return rc;
    }
    CK(launch_k(t.pdl && c->pdl(), k_loss_terms, (unsigned)(nG + ns), 256, 0, c->stream, x));
    return NEP_OK;
}

int launch_loss_final(Ctx *c, double *loss3, const double *fpart, int nf, const double *spart, int nsb, double nsv) {
    k_loss_final<<<1, 256, 0, c->stream>>>(fpart, nf, spart, nsb, c->n_sv.as<int>(), nsv, c->norm_Ns(), c->norm_Na(),
                                           loss3, c->gb1.as<double>());
    CK_LAUNCH("k_loss_final");
    return NEP_OK;
}

int launch_cotangents(Ctx *c, const double *dE, const float *dF, const double *dW) {
    if (c->n_atoms > 0) {
        k_fbar_rows<<<(unsigned)((c->n_atoms + 255) / 256), 256, 0, c->stream>>>(c->n_atoms, dF, c->fbar.as<float4>());
        CK_LAUNCH("k_fbar_rows");
    }
    k_cotangents<<<1, 256, 0, c->stream>>>(c->n_struct, c->atom_off.as<int64_t>(), dE, dW, c->ebar.as<float>(),
                                           c->wbar.as<float>(), c->gb1.as<double>());
    CK_LAUNCH("k_cotangents");
    return NEP_OK;
}

static size_t ann_smem(Ctx *c) {  // two buffers of staged rows
    const int NNP = (c->NN + 3) & ~3, NDQ = (c->NDP + 3) & ~3;
    return 2 * sizeof(float) * ANN_ROWS * (3 * NNP + 2 * NDQ);
}
// threads per block: the output tiles (whole warps, at most 256), and at least the neurons
// (the b0 / w1 sums of the first block take one thread per neuron)
static int ann_threads(Ctx *c) {
    const int ntiles = ((c->NN + 3) / 4) * ((c->NDP + 3) / 4);
    const int t = std::max((ntiles + 31) / 32 * 32, (c->NN + 31) / 32 * 32);
    return std::min(ANN_MAX_THREADS, t);
}
static int ann_groups(Ctx *c) {
    const int ntiles = ((c->NN + 3) / 4) * ((c->NDP + 3) / 4);
    return (ntiles + ann_threads(c) - 1) / ann_threads(c);
}

int prepare_loss_kernels(Ctx *c) {
    int maxo = 0;
    CK(cudaDeviceGetAttribute(&maxo, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    CK(cudaFuncSetAttribute(k_ann_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
    return NEP_OK;
}

int launch_ann_grad_chunks(Ctx *c, const int *chunks, int n_chunks) {
    if (n_chunks <= 0) return NEP_OK;
    CK(launch_k(c->pdl(), k_ann_grad, dim3(n_chunks, ann_groups(c)), ann_threads(c), ann_smem(c), c->stream, chunks,
                c->NN, c->NDP, c->zt.as<float>(), c->ut.as<float>(), c->om.as<float>(), c->st_qt.as<float>(),
                c->dqt.as<float>(), c->annpart.as<float>()));
    return NEP_OK;
}

int launch_ann_grad(Ctx *c) { return launch_ann_grad_chunks(c, c->chunk_begin.as<int>(), c->n_chunks); }

static int run_grad_final(Ctx *c, const GradArgs &g, bool pdl) {
    CK(launch_k(pdl, k_grad_reduce, dim3((unsigned)((c->P + 31) / 32), GF_SEG), dim3(32, GF_RG), 0, c->stream, g,
                c->gpart.as<float2>()));
    return NEP_OK;
}

static GradArgs grad_args(Ctx *c, float *grad) {
    GradArgs g;
    g.T = c->T;
    g.NN = c->NN;
    g.ND = c->ND;
    g.NDP = c->NDP;
    g.nR = c->nR;
    g.kR = c->kR;
    g.nA = c->nA;
    g.kA = c->kA;
    g.NRP = c->ks->NR;
    g.KRP = c->ks->KR;
    g.NAP = c->ks->NA;
    g.KAP = c->ks->KA;
    g.P = c->P;
    g.desc_map = c->d_desc_map.as<int>();
    g.annpart = c->annpart.as<float>();
    g.clo = c->type_clo.as<int>();
    g.chi = c->type_chi.as<int>();
    g.cpart = c->cpart.as<float>();
    g.wlo = c->adj.type_wlo.as<int>();
    g.whi = c->adj.type_whi.as<int>();
    g.warp_begin = c->adj.warp_begin.as<int>();
    g.gb1 = c->gb1.as<double>();
    g.grad = grad;
    g.acc = nullptr;
    g.counters = c->counters.as<unsigned>() + 2;
    g.opt = 0;
    return g;
}

int launch_grad_final_sched(Ctx *c, float *grad, const int *clo, const int *chi, const int *wlo, const int *whi,
                            const int *warp_begin, bool opt, const double *loss3, double lE, double lF, double lV) {
    GradArgs g = grad_args(c, grad);
    g.clo = clo;
    g.chi = chi;
    g.wlo = wlo;
    g.whi = whi;
    g.warp_begin = warp_begin;
    if (opt) {
        g.opt = 1;
        g.o = opt_args(c, loss3, lE, lF, lV, nullptr);
    }
    return run_grad_final(c, g, c->pdl());
}

int launch_grad_final(Ctx *c, float *grad, bool opt, const double *loss3, double lE, double lF, double lV) {
    GradArgs g = grad_args(c, grad);
    if (opt) {
        g.opt = 1;
        g.o = opt_args(c, loss3, lE, lF, lV, nullptr);
    }
    return run_grad_final(c, g, c->pdl());
}

// ----------------------------------------------------------------------------- plain form
// The baseline the batched pass is measured against: the same kernels and arithmetic,
// launched once per structure with one warp per atom, no CUDA graph, no multi-structure
// persistent schedule; the gradient of each structure is added to an FP64 accumulator.

static int build_plain(Ctx *c) {
    const int64_t ns = c->n_struct, na = c->n_atoms;
    const int T = c->T;
    std::vector<int> work(na), ident(na + 1), wlo(ns * T, 0), whi(ns * T, -1), clo(ns * T, 0), chi(ns * T, 0), cb;
    std::vector<int64_t> cofs(ns + 1, 0);
    int64_t maxn = 0;
    for (int64_t k = 0; k <= na; ++k) ident[k] = (int)k;
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t a0 = c->h_atom_off[s], a1 = c->h_atom_off[s + 1];
        maxn = std::max(maxn, a1 - a0);
        std::vector<int> at;
        for (int64_t i = a0; i < a1; ++i) at.push_back((int)i);
        std::stable_sort(at.begin(), at.end(), [&](int x, int y) { return c->h_type[x] < c->h_type[y]; });
        for (size_t k = 0; k < at.size(); ++k) work[a0 + k] = at[k];
        cofs[s] = (int64_t)cb.size();
        int64_t p = a0;
        for (int t = 0; t < T; ++t) {
            const int64_t q0 = p;
            while (p < a1 && c->h_type[work[p]] == t) ++p;
            clo[s * T + t] = (int)(cb.size() - cofs[s]);
            for (int64_t q = q0; q < p; q += 512) cb.push_back((int)q);
            chi[s * T + t] = (int)(cb.size() - cofs[s]);
            if (p > q0) {
                wlo[s * T + t] = (int)(q0 - a0);
                whi[s * T + t] = (int)(p - 1 - a0);
            }
        }
        cb.push_back((int)a1);  // closes the last chunk of s (not a chunk start of s + 1)
    }
    cofs[ns] = (int64_t)cb.size();
    c->p_cofs = cofs;
    if (c->p_work.ensure<int>(na) || c->p_ident.ensure<int>(na + 1) || c->p_wlo.ensure<int>(ns * T) ||
        c->p_whi.ensure<int>(ns * T) || c->p_clo.ensure<int>(ns * T) || c->p_chi.ensure<int>(ns * T) ||
        c->p_chunks.ensure<int>((int64_t)cb.size() + 1) || c->p_acc.ensure<double>(c->P) ||
        c->p_part.ensure<double>(ns * 5 + 8))
        return c->fail(NEP_ENOMEM, "plain-form buffers");
    const int NC = c->ks->NR * c->ks->KR + c->ks->NA * c->ks->KA;
    if (c->cpart.bytes < sizeof(float) * (size_t)(maxn + T) * T * NC &&
        c->cpart.ensure<float>((int64_t)std::max<int64_t>(maxn, c->adj.W) * T * NC + (int64_t)T * T * NC))
        return c->fail(NEP_ENOMEM, "plain-form partials");
    CK(cudaMemcpy(c->p_work.ptr, work.data(), sizeof(int) * na, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_ident.ptr, ident.data(), sizeof(int) * (na + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_wlo.ptr, wlo.data(), sizeof(int) * ns * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_whi.ptr, whi.data(), sizeof(int) * ns * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_clo.ptr, clo.data(), sizeof(int) * ns * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_chi.ptr, chi.data(), sizeof(int) * ns * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->p_chunks.ptr, cb.data(), sizeof(int) * cb.size(), cudaMemcpyHostToDevice));
    if (int rc = build_work_rec(c, c->p_work.as<int>(), c->p_rec, c->p_rec2)) return rc;
    c->plain_ready = true;
    return NEP_OK;
}

int run_plain_loss(Ctx *c, const double *Er, const float *Fr, const double *Wr, const uint8_t *hw, double lE,
                   double lF, double lV, double *loss3, float *grad) {
    int rc;
    if (!c->plain_ready && (rc = build_plain(c))) return rc;
    const int64_t ns = c->n_struct;
    const int GB = 2;  // gather blocks per structure
    double *pg = c->p_part.as<double>();
    double *ps = pg + ns * GB;
    if ((rc = launch_expand(c))) return rc;
    double nsv = c->ov_NsV > 0.0 ? c->ov_NsV : host_nsv(c, hw, 0, ns);
    if (nsv == 0.0) {  // counted once over the whole batch
        if ((rc = launch_count_hasw(c, hw, 0, ns))) return rc;
        nsv = -1.0;
    }
    CK(cudaMemsetAsync(c->p_acc.ptr, 0, sizeof(double) * c->P, c->stream));
    const int pv = 2;  // one warp per atom: lanes-per-atom 16, 128-register variant
    const size_t gsm = ann_smem(c);
    const int groups = ann_groups(c);
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t a0 = c->h_atom_off[s], n = c->h_atom_off[s + 1] - a0;
        AtomArgs a = atom_args(c);
        a.work = c->p_work.as<int>();
        a.rec = c->p_rec.as<int4>();
        a.rec2 = c->p_rec2.as<int2>();
        a.warp_begin = c->p_ident.as<int>() + a0;
        const int nch = (int)(c->p_cofs[s + 1] - c->p_cofs[s] - 1);
        a.chunks = c->p_chunks.as<int>() + c->p_cofs[s];
        a.n_chunks = nch;
        a.chunk_rows = 512;
        c->ks->launch_fwd[pv](a, (int)n, 1, -1, c->stream, false);
        CK_LAUNCH("forward stages (plain)");
        TermsCall t;
        t.a0 = a0;
        t.a1 = a0 + n;
        t.s0 = s;
        t.s1 = s + 1;
        t.F_out = c->F_int.as<float>();
        t.E_out = c->E_int.as<double>();
        t.W_out = c->W_int.as<double>();
        t.loss = true;
        t.F_ref = Fr;
        t.E_ref = Er;
        t.W_ref = Wr;
        t.has_W = hw;
        t.lE = lE;
        t.lF = lF;
        t.lV = lV;
        t.nsv = nsv;
        t.fpart = pg + s * GB;
        t.spart = ps + 3 * s;
        t.gather_blocks = GB;
        t.pdl = false;
        if ((rc = launch_terms(c, t))) return rc;
        c->ks->launch_adj[pv](a, (int)n, 1, -1, c->stream, false);
        CK_LAUNCH("adjoint stages (plain)");
        if (nch > 0) {
            k_ann_grad<<<dim3(nch, groups), ann_threads(c), gsm, c->stream>>>(c->p_chunks.as<int>() + c->p_cofs[s], c->NN, c->NDP,
                                                                   c->zt.as<float>(), c->ut.as<float>(),
                                                                   c->om.as<float>(), c->st_qt.as<float>(),
                                                                   c->dqt.as<float>(), c->annpart.as<float>());
            CK_LAUNCH("k_ann_grad (plain)");
        }
        GradArgs g = grad_args(c, nullptr);
        g.clo = c->p_clo.as<int>() + s * c->T;
        g.chi = c->p_chi.as<int>() + s * c->T;
        g.wlo = c->p_wlo.as<int>() + s * c->T;
        g.whi = c->p_whi.as<int>() + s * c->T;
        g.warp_begin = c->p_ident.as<int>() + a0;
        g.acc = c->p_acc.as<double>();
        if ((rc = run_grad_final(c, g, false))) return rc;
    }
    if ((rc = launch_loss_final(c, loss3, pg, (int)(ns * GB), ps, (int)ns, nsv))) return rc;
    k_grad_convert<<<(unsigned)((c->P + 255) / 256), 256, 0, c->stream>>>(c->P, (int64_t)c->T * c->NN * c->ND +
                                                                          2 * (int64_t)c->T * c->NN,
                                                                          c->p_acc.as<double>(), c->gb1.as<double>(),
                                                                          grad);
    CK_LAUNCH("k_grad_convert");
    return NEP_OK;
}

int launch_range(Ctx *c, const float *q, float *qmin, float *qmax) {
    k_range<<<c->ND, 256, 0, c->stream>>>(c->n_atoms, c->NDP, c->ND, c->d_desc_map.as<int>(), q, qmin, qmax);
    CK_LAUNCH("k_range");
    return NEP_OK;
}

int launch_compact_q(Ctx *c, const float *qp, float *q) {
    const int64_t n = c->n_atoms * c->ND;
    if (n == 0) return NEP_OK;
    k_compact_q<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->n_atoms, c->NDP, c->ND,
                                                                     c->d_desc_map.as<int>(), qp, q);
    CK_LAUNCH("k_compact_q");
    return NEP_OK;
}

}  // namespace nep
