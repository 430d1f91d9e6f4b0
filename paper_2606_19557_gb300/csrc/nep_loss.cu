// Force gather, per-structure sums, the E/F/W loss, and the deterministic reductions
// of the parameter gradient (hot-path steps a5-a7 and the reduction halves of a9/a10).
//
// Fixed-order reductions everywhere: per-warp FP64 sums in a fixed lane order, per-block
// partials in a fixed warp order, and a final pass over the partials in index order.
// No floating-point atomics, so two runs with the same launch shape are bit-identical.
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

// --------------------------------------------------------------------------- forces
// F_i = sum_{p in N(i)} G_p - sum_{p in N(i)} G_{rev(p)}: the second sum visits the pairs
// (j, i, -S) of which i is the neighbour, through the reverse index (no atomics).
__global__ void k_gather(int64_t a0, int64_t a1, const int64_t *nbr_off, const int *rev, const float4 *G,
                         const float *F_own, float *F_out, const float *F_ref, float coefF, int loss, float *fbar,
                         double *part) {
    __shared__ double wpart[32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * nw + wib, W = (int64_t)gridDim.x * nw;
    double acc = 0.0;
    for (int64_t i = a0 + gw; i < a1; i += W) {
        const int64_t beg = nbr_off[i], end = nbr_off[i + 1];
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for (int64_t p0 = beg; p0 < end; p0 += 128) {  // 4 index loads, then 4 gathers, in flight
            int r[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t p = p0 + lane + 32 * k;
                r[k] = p < end ? rev[p] : -1;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (r[k] >= 0) {
                    const float4 g = G[r[k]];
                    sx += g.x;
                    sy += g.y;
                    sz += g.z;
                }
            }
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        sz = warp_sum(sz);
        if (lane < 3) {
            const float own = F_own[i * 3 + lane];
            const float F = own - (lane == 0 ? sx : lane == 1 ? sy : sz);
            F_out[i * 3 + lane] = F;
            if (loss) {
                const float d = F - F_ref[i * 3 + lane];
                fbar[i * 4 + lane] = coefF * d;  // float4 rows (x, y, z, unused)
                acc += (double)d * (double)d;
            }
        }
    }
    if (loss) {
        acc += __shfl_down_sync(FULL, acc, 1);
        acc += __shfl_down_sync(FULL, acc, 2);  // lanes 0..2 hold the sums; lane 0 gets 0+1+2(+3=0)
        if (lane == 0) wpart[wib] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < nw; ++k) s += wpart[k];
            part[blockIdx.x] = s;
        }
    }
}

// --------------------------------------------------------------------------- structures
// E_s = sum_i E_i and W_s = sum_i W_i in FP64 (Eq. 1); loss terms and cotangents of Eq. "loss".
// One block per structure: its threads stride over the structure's atoms, then a fixed-order
// reduction (lanes, then warps in order), so a 10,000-atom cell is summed by 256 threads.
// The block size (~4 atoms per thread, from the launch's mean structure size) fixes the
// summation order.  part[3 * (s - s0) + q]: the structure's loss terms.
__global__ void k_struct(int64_t s0, int64_t s1, const int64_t *atom_off, const float *E_atom, const float *W_atom,
                         double *E_out, double *W_out, int loss, const double *E_ref, const double *W_ref,
                         const uint8_t *has_W, const int *n_sv, double nsv_over, double lamE, double lamV, double Ns,
                         float *ebar, float *wbar, double *part /*[s1 - s0][3]*/) {
    __shared__ double red[32][10];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t s = s0 + blockIdx.x;
    if (s >= s1) return;
    const int64_t b = atom_off[s], e = atom_off[s + 1];
    double v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        v[0] += (double)E_atom[i];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[1 + k] += (double)W_atom[i * 9 + k];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = warp_sum_d(v[k]);
    if (lane == 0)
        for (int k = 0; k < 10; ++k) red[wib][k] = v[k];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double E = 0.0, Wv[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < nw; ++w) {
        E += red[w][0];
        for (int k = 0; k < 9; ++k) Wv[k] += red[w][1 + k];
    }
    E_out[s] = E;
    for (int k = 0; k < 9; ++k) W_out[s * 9 + k] = Wv[k];
    if (!loss) return;
    // FP64 division is slow on this part: one reciprocal per structure, coefficients once
    const double NsV = nsv_over > 0.0 ? nsv_over : (double)(*n_sv);
    const double na = (double)(e - b);
    const double inv_na = 1.0 / na, inv_na2 = inv_na * inv_na;
    const double dE = E - E_ref[s];
    const double aE = (dE * inv_na) * (dE * inv_na);
    const double eb = (lamE * 2.0 / Ns) * dE * inv_na2;
    ebar[s] = (float)eb;
    const double ab1 = -na * eb;
    double aV = 0.0;
    const bool hw = has_W == nullptr || has_W[s] != 0;
    const double cV = NsV > 0.0 ? lamV * 2.0 / (9.0 * NsV) : 0.0;
    for (int k = 0; k < 9; ++k) {
        double wb = 0.0;
        if (hw && NsV > 0.0) {
            const double dW = Wv[k] - W_ref[s * 9 + k];
            aV += (dW * inv_na) * (dW * inv_na);
            wb = cV * dW * inv_na2;
        }
        wbar[s * 9 + k] = (float)wb;
    }
    part[3 * (s - s0) + 0] = aE;
    part[3 * (s - s0) + 1] = aV;
    part[3 * (s - s0) + 2] = ab1;
}

__global__ void k_count_hasw(int64_t ns, const uint8_t *has_W, int *n_sv) {
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

__global__ void k_loss_final(const double *fpart, int nf, const double *spart, int nsb, const int *n_sv,
                             double nsv_over, double Ns, double Na, double *loss3, double *gb1) {
    __shared__ double sh[4][256];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nsb; k += blockDim.x) {
        a[0] += spart[3 * k];
        a[2] += spart[3 * k + 1];
        a[3] += spart[3 * k + 2];
    }
    for (int k = threadIdx.x; k < nf; k += blockDim.x) a[1] += fpart[k];
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nsv = nsv_over > 0.0 ? nsv_over : (double)(*n_sv);
        loss3[0] = Ns > 0 ? sh[0][0] / Ns : 0.0;
        loss3[1] = Na > 0 ? sh[1][0] / (3.0 * Na) : 0.0;
        loss3[2] = nsv > 0 ? sh[2][0] / (9.0 * nsv) : 0.0;
        *gb1 = sh[3][0];
    }
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
// block per chunk of work positions holding a single species; each thread accumulates
// a 4 x 4 register tile of the NN x ND output; FP32 partial per chunk.
constexpr int ANN_ROWS = 32;
constexpr int ANN_TILES = 128;  // 4x4 tiles per block (blockIdx.y covers the rest)

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
    extern __shared__ __align__(16) float sm[];
    const int NNP = (NN + 3) & ~3, NDQ = (NDP + 3) & ~3;
    const int tile_floats = ANN_ROWS * (3 * NNP + 2 * NDQ);
    const AnnTile buf[2] = {ann_tile(sm, NNP, NDQ), ann_tile(sm + tile_floats, NNP, NDQ)};
    const int c = blockIdx.x;
    const int r0 = chunk_begin[c], r1 = chunk_begin[c + 1];
    const int tn = NDQ / 4, ntiles = (NNP / 4) * tn;
    const int tile = blockIdx.y * ANN_TILES + threadIdx.x;
    const bool own = threadIdx.x < ANN_TILES && tile < ntiles;
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
};

// Two passes.  k_grad_part: one block per (32 consecutive parameters, row segment), with
// GF_RG row groups (threadIdx.y); the threads of a warp read 32 neighbouring parameters of
// one partial row (coalesced), each thread keeps four FP64 chains, the row groups are added
// in a fixed order and each segment's sum goes to gpart[seg][k].  k_grad_sum adds the
// GF_SEG segments of each parameter in order.  Spreading the rows over segments keeps
// every SM busy with the FP64 additions.
constexpr int GF_RG = 32;
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

__global__ void k_grad_part(GradArgs g, double *gpart /*[GF_SEG][P]*/) {
    __shared__ double red[GF_RG][33];
    const int tx = threadIdx.x, ty = threadIdx.y, seg = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * 32 + tx;
    const int T = g.T, NC = g.NRP * g.KRP + g.NAP * g.KAP;
    const int annstride = g.NN * g.NDP + 2 * g.NN;
    double s = 0.0;
    if (k < g.P) {
        const GradSource r = grad_source(g, k);
        if (!r.b1) {
            const int len = (r.hi - r.lo + GF_SEG - 1) / GF_SEG;
            const int lo = r.lo + seg * len, hi = min(r.hi, lo + len);
            double s4[4] = {0.0, 0.0, 0.0, 0.0};  // four independent chains keep four loads in flight
            int q = 0;
            if (r.net) {
                for (int c = lo + ty; c < hi; c += GF_RG, q = (q + 1) & 3)
                    s4[q] += (double)g.annpart[(size_t)c * annstride + r.off];
            } else {
                for (int w = lo + ty; w < hi; w += GF_RG, q = (q + 1) & 3)
                    if (g.warp_begin[w] < g.warp_begin[w + 1])
                        s4[q] += (double)g.cpart[((size_t)(w + r.a) * T + r.b) * NC + r.off];
            }
            s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
    }
    red[ty][tx] = s;
    __syncthreads();
    if (ty != 0 || k >= g.P) return;
    double tot = 0.0;
    for (int rr = 0; rr < GF_RG; ++rr) tot += red[rr][tx];
    gpart[(size_t)seg * g.P + k] = tot;
}

__global__ void k_grad_sum(GradArgs g, const double *gpart) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.P) return;
    const GradSource r = grad_source(g, k);
    double tot = 0.0;
    for (int seg = 0; seg < GF_SEG; ++seg) tot += gpart[(size_t)seg * g.P + k];
    if (r.b1) tot = g.acc ? 0.0 : *g.gb1;
    if (g.acc) g.acc[k] += r.sign * tot;
    else g.grad[k] = (float)(r.sign * tot);
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
    a.NDP = c->NDP;
    a.st_D = c->st_D.as<float>();
    a.st_S = c->st_S.as<float>();
    a.st_b = c->st_b.as<float>();
    a.st_ab = c->st_ab.as<float>();
    a.st_E = c->st_E.as<float>();
    return a;
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
    k_expand<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(x);
    CK_LAUNCH("k_expand");
    return NEP_OK;
}

int launch_forward(Ctx *c, float *q_raw, int stage) {
    if (c->n_atoms == 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.warp_begin = c->fwd.warp_begin.as<int>();
    a.q_raw = q_raw;
    c->ks->launch_fwd[c->fwd.var](a, c->fwd.blocks, c->fwd.wpb, stage, c->stream);
    CK_LAUNCH("forward stages");
    return NEP_OK;
}

int launch_adjoint(Ctx *c, int stage) {
    if (c->n_atoms == 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.warp_begin = c->adj.warp_begin.as<int>();
    c->ks->launch_adj[c->adj.var](a, c->adj.blocks, c->adj.wpb, stage, c->stream);
    CK_LAUNCH("adjoint stages");
    return NEP_OK;
}

int launch_forward_sched(Ctx *c, const int *work, const int *warp_begin, int blocks, int var, int wpb,
                         const int *chunks, int n_chunks) {
    if (blocks <= 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.work = work;
    a.warp_begin = warp_begin;
    a.chunks = chunks;
    a.n_chunks = n_chunks;
    c->ks->launch_fwd[var](a, blocks, wpb, -1, c->stream);
    CK_LAUNCH("forward stages");
    return NEP_OK;
}

int launch_adjoint_sched(Ctx *c, const int *work, const int *warp_begin, int blocks, int var, int wpb,
                         const int *chunks, int n_chunks) {
    if (blocks <= 0) return NEP_OK;
    AtomArgs a = atom_args(c);
    a.work = work;
    a.warp_begin = warp_begin;
    a.chunks = chunks;
    a.n_chunks = n_chunks;
    c->ks->launch_adj[var](a, blocks, wpb, -1, c->stream);
    CK_LAUNCH("adjoint stages");
    return NEP_OK;
}

static int gather_blocks(Ctx *c) { return c->n_sm * 4; }


int launch_gather(Ctx *c, float *F_out, const float *F_ref, double lamF, bool loss, int64_t a0, int64_t a1,
                  double *part, int nblocks) {
    if (a1 <= a0) return NEP_OK;
    const int nb = nblocks > 0 ? nblocks : gather_blocks(c);
    const float coef = (float)(lamF * 2.0 / (3.0 * c->norm_Na()));
    k_gather<<<nb, 256, 0, c->stream>>>(a0, a1, c->nbr_off.as<int64_t>(), c->rev.as<int>(), (const float4 *)c->G.ptr,
                                        c->F_own.as<float>(), F_out, F_ref, coef, loss ? 1 : 0, c->fbar.as<float>(),
                                        part ? part : c->loss_part.as<double>());
    CK_LAUNCH("k_gather");
    return NEP_OK;
}

int launch_count_hasw(Ctx *c, const uint8_t *has_W, int64_t s0, int64_t s1) {
    if (s1 < 0) s1 = c->n_struct;
    k_count_hasw<<<1, 256, 0, c->stream>>>(s1 - s0, has_W ? has_W + s0 : nullptr, c->n_sv.as<int>());
    CK_LAUNCH("k_count_hasw");
    return NEP_OK;
}

static int64_t pow2ceil_host(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

int launch_struct(Ctx *c, double *E_out, double *W_out, const double *E_ref, const double *W_ref,
                  const uint8_t *has_W, double lamE, double lamV, bool loss, int64_t s0, int64_t s1, double *part,
                  int nblocks) {
    if (s1 <= s0) return NEP_OK;
    (void)nblocks;  // one block per structure, ~4 atoms per thread (32 to 256 threads)
    c->struct_parts = s1 - s0;
    const int64_t mean = (c->h_atom_off[s1] - c->h_atom_off[s0]) / (s1 - s0);
    const int threads = (int)std::min<int64_t>(256, std::max<int64_t>(32, pow2ceil_host(mean / 4)));
    k_struct<<<(unsigned)(s1 - s0), threads, 0, c->stream>>>(s0, s1, c->atom_off.as<int64_t>(), c->E_atom.as<float>(),
                                        c->W_atom.as<float>(), E_out, W_out, loss ? 1 : 0, E_ref, W_ref, has_W,
                                        c->n_sv.as<int>(), c->ov_NsV, lamE, lamV, c->norm_Ns(), c->ebar.as<float>(),
                                        c->wbar.as<float>(), part ? part : c->loss_part.as<double>() + gather_blocks(c));
    CK_LAUNCH("k_struct");
    return NEP_OK;
}

int launch_loss_final(Ctx *c, double *loss3, const double *fpart, int nf, const double *spart, int nsb) {
    if (!fpart) {
        fpart = c->loss_part.as<double>();
        nf = c->n_atoms > 0 ? gather_blocks(c) : 0;
        spart = c->loss_part.as<double>() + gather_blocks(c);
        nsb = c->n_struct > 0 ? (int)c->struct_parts : 0;
    }
    k_loss_final<<<1, 256, 0, c->stream>>>(fpart, nf, spart, nsb, c->n_sv.as<int>(), c->ov_NsV, c->norm_Ns(),
                                           c->norm_Na(), loss3, c->gb1.as<double>());
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
static int ann_groups(Ctx *c) {
    const int ntiles = ((c->NN + 3) / 4) * ((c->NDP + 3) / 4);
    return (ntiles + ANN_TILES - 1) / ANN_TILES;
}

int prepare_loss_kernels(Ctx *c) {
    int maxo = 0;
    CK(cudaDeviceGetAttribute(&maxo, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    CK(cudaFuncSetAttribute(k_ann_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
    return NEP_OK;
}

int launch_ann_grad(Ctx *c) {
    if (c->n_chunks == 0) return NEP_OK;
    k_ann_grad<<<dim3(c->n_chunks, ann_groups(c)), ANN_TILES, ann_smem(c), c->stream>>>(c->chunk_begin.as<int>(), c->NN, c->NDP, c->zt.as<float>(),
                                                      c->ut.as<float>(), c->om.as<float>(), c->st_qt.as<float>(),
                                                      c->dqt.as<float>(), c->annpart.as<float>());
    CK_LAUNCH("k_ann_grad");
    return NEP_OK;
}

int launch_ann_grad_chunks(Ctx *c, const int *chunks, int n_chunks) {
    if (n_chunks <= 0) return NEP_OK;
    k_ann_grad<<<dim3(n_chunks, ann_groups(c)), ANN_TILES, ann_smem(c), c->stream>>>(
        chunks, c->NN, c->NDP, c->zt.as<float>(), c->ut.as<float>(), c->om.as<float>(), c->st_qt.as<float>(),
        c->dqt.as<float>(), c->annpart.as<float>());
    CK_LAUNCH("k_ann_grad");
    return NEP_OK;
}

static int run_grad_final(Ctx *c, const GradArgs &g) {
    double *gp = c->gpart.as<double>();
    k_grad_part<<<dim3((unsigned)((c->P + 31) / 32), GF_SEG), dim3(32, GF_RG), 0, c->stream>>>(g, gp);
    CK_LAUNCH("k_grad_part");
    k_grad_sum<<<(unsigned)((c->P + 255) / 256), 256, 0, c->stream>>>(g, gp);
    CK_LAUNCH("k_grad_sum");
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
    return g;
}

int launch_grad_final_sched(Ctx *c, float *grad, const int *clo, const int *chi, const int *wlo, const int *whi,
                            const int *warp_begin) {
    GradArgs g = grad_args(c, grad);
    g.clo = clo;
    g.chi = chi;
    g.wlo = wlo;
    g.whi = whi;
    g.warp_begin = warp_begin;
    return run_grad_final(c, g);
}

int launch_grad_final(Ctx *c, float *grad) {
    GradArgs g = grad_args(c, grad);
    return run_grad_final(c, g);
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
    if ((rc = launch_count_hasw(c, hw))) return rc;
    CK(cudaMemsetAsync(c->p_acc.ptr, 0, sizeof(double) * c->P, c->stream));
    const int pv = 2;  // one warp per atom: lanes-per-atom 16, 128-register variant
    const size_t gsm = ann_smem(c);
    const int groups = ann_groups(c);
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t a0 = c->h_atom_off[s], n = c->h_atom_off[s + 1] - a0;
        AtomArgs a = atom_args(c);
        a.work = c->p_work.as<int>();
        a.warp_begin = c->p_ident.as<int>() + a0;
        const int nch = (int)(c->p_cofs[s + 1] - c->p_cofs[s] - 1);
        a.chunks = c->p_chunks.as<int>() + c->p_cofs[s];
        a.n_chunks = nch;
        c->ks->launch_fwd[pv](a, (int)n, 1, -1, c->stream);
        CK_LAUNCH("forward stages (plain)");
        if ((rc = launch_gather(c, c->F_int.as<float>(), Fr, lF, true, a0, a0 + n, pg + s * GB, GB))) return rc;
        if ((rc = launch_struct(c, c->E_int.as<double>(), c->W_int.as<double>(), Er, Wr, hw, lE, lV, true, s, s + 1,
                                ps + s * 3, 1)))
            return rc;
        c->ks->launch_adj[pv](a, (int)n, 1, -1, c->stream);
        CK_LAUNCH("adjoint stages (plain)");
        if (nch > 0) {
            k_ann_grad<<<dim3(nch, groups), ANN_TILES, gsm, c->stream>>>(c->p_chunks.as<int>() + c->p_cofs[s], c->NN, c->NDP,
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
        if ((rc = run_grad_final(c, g))) return rc;
    }
    if ((rc = launch_loss_final(c, loss3, pg, (int)(ns * GB), ps, (int)ns))) return rc;
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
