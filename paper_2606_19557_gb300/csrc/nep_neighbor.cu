// Cell-list neighbour search emitting CSR neighbour lists (kept on the GPU, Sec. "Training
// efficiency").
//
// The paper builds neighbour lists and displacement vectors once and keeps them on
// the GPU (Sec. "Training efficiency ..."); this file does the same for a whole
// batch of periodic, possibly triclinic, structures:
//   1. per structure: inverse cell, plane spacings w_a = V/|b x c| (FP64), bins per
//      axis n_a = max(1, floor(w_a / (rc + skin))) and scan reach m_a = ceil((rc + skin) n_a / w_a);
//   2. per atom: fractional coordinates, wrap offset, bin; counting sort into bins;
//   3. per atom (one warp): scan the candidates, either the (2 m_a + 1) neighbouring
//      bin images or, for a structure held in one bin per axis, each atom's own box of
//      periodic images; count the pairs and keep the 64-bit keys (group, t_j, j, S) of
//      up to `cap` of them (a second scan writes the keys only if some atom has more);
//   4. per atom (one warp): rank-sort its keys, decode to the float4 pair record;
//   5. per pair: index of the reverse pair (j, i, -S) by binary search.
// Pair predicate (identical here, in the oracle's brute force and in the per-atom
// kernels): d = ((double)r_j - (double)r_i) + S.h evaluated in double without fused
// multiply-add, rounded once to float; kept iff float (dx*dx + dy*dy) + dz*dz < rc*rc.
// Negating S negates every operation exactly, so d(j,i,-S) = -d(i,j,S) bit for bit
// and the radial/angular lists are symmetric.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nep_ctx.cuh"

namespace nep {

// ----------------------------------------------------------------------------- scan

namespace {

__global__ void k_scan_blocks(const int64_t *in, int64_t n, int64_t *block_sum) {
    __shared__ int64_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * 1024;
    int64_t s = 0;
    for (int k = 0; k < 4; ++k) {
        const int64_t idx = base + threadIdx.x * 4 + k;
        if (idx < n) s += in[idx];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_tot[w];
        block_sum[blockIdx.x] = t;
    }
}

__global__ void k_scan_sums(int64_t *block_sum, int64_t nb, int64_t *total) {
    // single block of 1024 threads, exclusive scan in chunks with a carry
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
        const int64_t idx = c0 + threadIdx.x;
        const int64_t v = idx < nb ? block_sum[idx] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const int64_t before = (wid > 0 ? warp_tot[wid - 1] : 0) + carry;
        if (idx < nb) block_sum[idx] = before + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int64_t *in, int64_t n, const int64_t *block_off, int64_t *out) {
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
    int64_t v[4];
    int64_t s = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t run = block_off[blockIdx.x] + (wid > 0 ? warp_tot[wid - 1] : 0) + x - s;
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

}  // namespace

// Exclusive scan of in[0..n) into out[0..n], out[n] = total (out may alias nothing).
// The total is also left in *total_dev.
int scan_exclusive(Ctx *c, const int64_t *in, int64_t n, int64_t *out, int64_t *total_dev) {
    if (n == 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
        CK(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), c->stream));
        return NEP_OK;
    }
    const int64_t nb = (n + 1023) / 1024;
    if (c->scan_tmp.ensure<int64_t>(nb + 1) != NEP_OK) return c->fail(NEP_ENOMEM, "scan workspace");
    int64_t *bs = c->scan_tmp.as<int64_t>();
    k_scan_blocks<<<(unsigned)nb, 256, 0, c->stream>>>(in, n, bs);
    k_scan_sums<<<1, 1024, 0, c->stream>>>(bs, nb, total_dev);
    k_scan_apply<<<(unsigned)nb, 256, 0, c->stream>>>(in, n, bs, out);
    CK(cudaGetLastError());
    return NEP_OK;
}

// ----------------------------------------------------------------------------- geometry

namespace {

constexpr double SKIN = 1e-3;  // Angstrom of extra reach for binning (rounding margin)
constexpr int NBIN_MAX = 128;  // bins per axis and structure
constexpr int SMAX = 127;      // |S_a| limit of the packed shift

struct SGeom {
    double h[9];
    double inv[9];
    float hf[9];    // h as given (floats)
    float invf[9];  // inv rounded to float
    float nb[3];    // |b_a|, the norms of the columns of inv (reciprocal vectors), in float
    int n[3];
    int m[3];
};

__device__ __forceinline__ void atomic_err(int *err, int code) { atomicCAS(err, 0, code); }

__global__ void k_struct_geom(int64_t ns, const float *cell, double rc, SGeom *geom, int64_t *nbins, int *err) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    SGeom g;
    for (int k = 0; k < 9; ++k) {
        g.hf[k] = cell[9 * s + k];
        g.h[k] = (double)cell[9 * s + k];
    }
    const double *h = g.h;
    const double c0[3] = {h[4] * h[8] - h[5] * h[7], h[5] * h[6] - h[3] * h[8], h[3] * h[7] - h[4] * h[6]};
    const double c1[3] = {h[7] * h[2] - h[8] * h[1], h[8] * h[0] - h[6] * h[2], h[6] * h[1] - h[7] * h[0]};
    const double c2[3] = {h[1] * h[5] - h[2] * h[4], h[2] * h[3] - h[0] * h[5], h[0] * h[4] - h[1] * h[3]};
    const double vol = h[0] * c0[0] + h[1] * c0[1] + h[2] * c0[2];
    if (!(fabs(vol) > 1e-9) || !isfinite(vol)) {
        atomic_err(err, 1);
        nbins[s] = 1;
        g.n[0] = g.n[1] = g.n[2] = 1;
        g.m[0] = g.m[1] = g.m[2] = 0;
        geom[s] = g;
        return;
    }
    for (int x = 0; x < 3; ++x) {
        g.inv[3 * x + 0] = c0[x] / vol;
        g.inv[3 * x + 1] = c1[x] / vol;
        g.inv[3 * x + 2] = c2[x] / vol;
    }
    for (int k = 0; k < 9; ++k) g.invf[k] = (float)g.inv[k];
    for (int a = 0; a < 3; ++a)
        g.nb[a] = (float)sqrt(g.inv[a] * g.inv[a] + g.inv[3 + a] * g.inv[3 + a] + g.inv[6 + a] * g.inv[6 + a]);
    const double w[3] = {fabs(vol) / sqrt(c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]),
                         fabs(vol) / sqrt(c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]),
                         fabs(vol) / sqrt(c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2])};
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) {
        int n = (int)floor(w[a] / (rc + SKIN));
        n = n < 1 ? 1 : (n > NBIN_MAX ? NBIN_MAX : n);
        const int m = (int)ceil((rc + SKIN) * n / w[a]);
        if (m > SMAX - 2) atomic_err(err, 2);
        g.n[a] = n;
        g.m[a] = m > SMAX - 2 ? SMAX - 2 : m;
        nb *= n;
    }
    geom[s] = g;
    nbins[s] = nb;
}

__global__ void k_struct_of(int64_t ns, const int64_t *atom_off, int *struct_of) {
    const int64_t s = blockIdx.x;
    if (s >= ns) return;
    for (int64_t i = atom_off[s] + threadIdx.x; i < atom_off[s + 1]; i += blockDim.x) struct_of[i] = (int)s;
}

__global__ void k_atom_bin(int64_t na, const float *pos, const int *type, int T, const int *struct_of,
                           const SGeom *geom, const int64_t *bin_off, int64_t *atom_bin, int4 *atom_wrap,
                           int64_t *bin_cnt, float4 *pos4, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int t = type[i];
    if (t < 0 || t >= T) atomic_err(err, 3);
    pos4[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], __int_as_float(t & 15));
    const int s = struct_of[i];
    const SGeom &g = geom[s];
    const double p[3] = {(double)pos[3 * i], (double)pos[3 * i + 1], (double)pos[3 * i + 2]};
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) {
        atomic_err(err, 4);
        atom_bin[i] = bin_off[s];
        atom_wrap[i] = make_int4(0, 0, 0, 0);
        atomicAdd((unsigned long long *)&bin_cnt[bin_off[s]], 1ull);
        return;
    }
    int b[3], wr[3];
    for (int a = 0; a < 3; ++a) {
        const double f = p[0] * g.inv[0 * 3 + a] + p[1] * g.inv[1 * 3 + a] + p[2] * g.inv[2 * 3 + a];
        const double fl = floor(f);
        const double fw = f - fl;
        int bb = (int)(fw * g.n[a]);
        bb = bb < 0 ? 0 : (bb >= g.n[a] ? g.n[a] - 1 : bb);
        b[a] = bb;
        if (fabs(fl) > 1e6) atomic_err(err, 4);
        wr[a] = (int)fl;
    }
    const int64_t bin = bin_off[s] + ((int64_t)b[0] * g.n[1] + b[1]) * g.n[2] + b[2];
    atom_bin[i] = bin;
    atom_wrap[i] = make_int4(wr[0], wr[1], wr[2], 0);
    atomicAdd((unsigned long long *)&bin_cnt[bin], 1ull);
}

__global__ void k_bin_fill(int64_t na, const int64_t *atom_bin, const int64_t *bin_start, int64_t *bin_cur,
                           int *bin_atoms) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int64_t bin = atom_bin[i];
    const int64_t slot = (int64_t)atomicAdd((unsigned long long *)&bin_cur[bin], 1ull);
    bin_atoms[bin_start[bin] + slot] = (int)i;
}

// The atoms of every bin in bin order: (x, y, z, bits(j << 4 | t_j)) and the wrap offsets,
// so that the lanes scanning a bin read consecutive entries and no species table.
__global__ void k_bin_pack(int64_t na, const int *bin_atoms, const float4 *pos4, const int4 *atom_wrap,
                           float4 *bin_pos, int4 *bin_wrap) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na) return;
    const int j = bin_atoms[t];
    const float4 p = pos4[j];
    bin_pos[t] = make_float4(p.x, p.y, p.z, __int_as_float((j << 4) | __float_as_int(p.w)));
    bin_wrap[t] = atom_wrap[j];
}

// The pair predicate.  Returns the float squared length; d32 receives the float displacement.
__device__ __forceinline__ float pair_d(const float *pi, const float *pj, const double *h, int Sa, int Sb, int Sc,
                                        float *d32) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const double rel = __dsub_rn((double)pj[x], (double)pi[x]);
        const double sh = __dadd_rn(__dadd_rn(__dmul_rn((double)Sa, h[x]), __dmul_rn((double)Sb, h[3 + x])),
                                    __dmul_rn((double)Sc, h[6 + x]));
        d32[x] = __double2float_rn(__dadd_rn(rel, sh));
    }
    return __fadd_rn(__fadd_rn(__fmul_rn(d32[0], d32[0]), __fmul_rn(d32[1], d32[1])), __fmul_rn(d32[2], d32[2]));
}

// Knuth's TwoSum: s + e = a + b exactly (round to nearest, no overflow).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// TwoProduct by a fused multiply-add (Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005): p + e = a b exactly when a b does not underflow.
__device__ __forceinline__ float two_prod(float a, float b, float &e) {
    const float p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
    return p;
}

// Exponent of the lowest set-able bit (unit in the last place) of a nonzero float.
__device__ __forceinline__ int lsb_exp(float v) {
    const int ev = (__float_as_int(v) >> 23) & 0xff;
    return (ev > 0 ? ev : 1) - 150;
}

// pair_d's displacement in FP32 arithmetic, for pairs with a periodic image.  Per
// component, X = (p_j - p_i) + S_a h_a + S_b h_b + S_c h_c is carried exactly as the
// float expansion h3 + (error terms) (TwoSum of the difference, TwoProduct of the image
// terms, TwoSum of the running sum), and c = RN(h3 + lo) with the exact remainder r.
// Bounds: |X - (c + r)| <= 6 2^-48 M (the float sum lo of seven error terms, each at
// most 2^-24 of its operand, M the sum of the operand magnitudes), and the FP64 form
// D of pair_d differs from X by at most 2^-53 (|p_j - p_i| + |S_a h_a + S_b h_b| +
// |sum of the image terms| + |D|) <= 2^-52 M + 2^-51 |c|.  With B >= both, if r + B and
// r - B stay inside half the float gaps above and below c, then X and D lie in the
// rounding interval of c, so fl32(D), the predicate's float, equals c.  Near a rounding
// boundary (an exact tie is common: X then has one bit more than a float) c is kept when
// nothing was rounded at all: lo's own sum is exact and every FP64 partial sum of pair_d
// is exact, because all operands are multiples of 2^q (q the lowest unit in the last
// place among them) and every partial sum is below M < 2^(q+52); then D = X = h3 + lo and
// c = RN(X) = fl32(D), ties to even included.  Returns false (the caller takes the FP64
// form) when neither can be shown, and for a zero or tiny c.
// An all-zero component is summed as the FP64 form associates it, so its zero sign
// follows the same IEEE rules.
__device__ __forceinline__ bool pair_d_fp32(const float *pi, const float *pj, const float *hf, int Sa, int Sb,
                                            int Sc, float *d32) {
    const float fa = (float)Sa, fb = (float)Sb, fc = (float)Sc;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        float e0, e1, e2, e3, t1, t2, t3, rr;
        const float s0 = two_sum(pj[x], -pi[x], e0);
        const float p1 = two_prod(fa, hf[x], e1);
        const float p2 = two_prod(fb, hf[3 + x], e2);
        const float p3 = two_prod(fc, hf[6 + x], e3);
        const float h1 = two_sum(s0, p1, t1);
        const float h2 = two_sum(h1, p2, t2);
        const float h3 = two_sum(h2, p3, t3);
        const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, e3)), __fadd_rn(__fadd_rn(t1, t2), t3));
        const float c = two_sum(h3, lo, rr);
        const float M = fabsf(s0) + fabsf(p1) + fabsf(p2) + fabsf(p3) + fabsf(h1) + fabsf(h2) + fabsf(h3);
        if (c == 0.0f) {
            if (M != 0.0f || lo != 0.0f || rr != 0.0f) return false;
            d32[x] = __fadd_rn(s0, __fadd_rn(__fadd_rn(p1, p2), p3));  // zeros, associated as in pair_d
            continue;
        }
        const int ec = (__float_as_int(c) >> 23) & 0xff;
        if (ec < 40 || ec == 255) return false;
        // half the gaps to the floats above and below |c| = 2^e (1 + m): 2^(e-24) each, except
        // below a power of two (m = 0), where the gap halves
        const float hg = __int_as_float((ec - 24) << 23);
        const float hg_small = (__float_as_int(c) & 0x7fffff) ? hg : __int_as_float((ec - 25) << 23);
        const float up = c > 0.0f ? hg : hg_small, down = c > 0.0f ? hg_small : hg;  // towards +inf / -inf
        const float B = 0x1p-44f * M + 0x1p-51f * fabsf(c) + 0x1p-110f;
        if (!(rr + B < up && rr - B > -down)) {
            float r1, r2, r3, r4, r5, r6;
            const float a1 = two_sum(e0, e1, r1), a2 = two_sum(e2, e3, r2), a3 = two_sum(a1, a2, r3);
            const float b1 = two_sum(t1, t2, r4), b2 = two_sum(b1, t3, r5);
            two_sum(a3, b2, r6);  // its sum is lo
            if (r1 != 0.0f || r2 != 0.0f || r3 != 0.0f || r4 != 0.0f || r5 != 0.0f || r6 != 0.0f) return false;
            int q = 1000;
            if (pj[x] != 0.0f) q = min(q, lsb_exp(pj[x]));
            if (pi[x] != 0.0f) q = min(q, lsb_exp(pi[x]));
            if (Sa != 0 && hf[x] != 0.0f) q = min(q, lsb_exp(hf[x]));
            if (Sb != 0 && hf[3 + x] != 0.0f) q = min(q, lsb_exp(hf[3 + x]));
            if (Sc != 0 && hf[6 + x] != 0.0f) q = min(q, lsb_exp(hf[6 + x]));
            const int eM = ((__float_as_int(M) >> 23) & 0xff) - 127;  // M < 2^(eM + 1)
            if (eM + 2 > q + 52) return false;
        }
        d32[x] = c;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_shift(int Sa, int Sb, int Sc) {
    return ((uint32_t)(Sa + 128) << 16) | ((uint32_t)(Sb + 128) << 8) | (uint32_t)(Sc + 128);
}

// Warp-cooperative candidate scan of atom i (one warp per atom).  Calls hit(j, t_j, Sa, Sb, Sc, ang)
// for every pair within rcR (ang: also within rcA), from any lane, in no particular order
// (the lists are sorted afterwards).  Two ways to enumerate candidates, chosen per structure:
//   * a structure held in one bin per axis (a cell narrower than 2 rc): the lanes take the
//     structure's atoms j and each enumerates only the periodic images S that can lie
//     within the cutoff of i, the box |d.b_a| <= rcq |b_a| around the nearest image
//     (b_a the reciprocal vectors, so |d.b_a| <= |d| |b_a|);
//   * otherwise the (2m+1)^3 neighbouring bins, the lanes taking the atoms of each bin.
// Each candidate is first evaluated in FP32 with explicit rounding: q = (p_j - p_i) + S.h and
// r2q = |q|^2.  Every FP32 step is within half an ulp, so |q_x - d_x| <= 7 2^-24 B_x with
// B_x = |p_j,x| + |p_i,x| + sum_k |S_k h_k,x| (d the predicate's displacement); the band
// uses 2^-20 B_x, more than twice that, and bounds |r2q - r2| by M (below).  Only a candidate
// whose r2q lies within M of rc^2 (rcR or rcA) takes the exact FP64 predicate, so the
// slow FP64 units see a tiny fraction of the candidates and every decision is the
// predicate's.
template <class Fn>
__device__ __forceinline__ void scan_atom_warp(int64_t i, int lane, const float *pos, const float4 *pos4,
                                               const int *struct_of,
                                               const int64_t *atom_off, const SGeom *geom, const int64_t *bin_off,
                                               const int64_t *atom_bin, const int4 *atom_wrap,
                                               const int64_t *bin_start, const float4 *bin_pos, const int4 *bin_wrap,
                                               float rc2R, float rc2A, float rcq2, float rcq, int *err, Fn hit) {
    const int s = struct_of[i];
    const SGeom &g = geom[s];
    const float *pi = pos + 3 * i;
    const float hf[9] = {g.hf[0], g.hf[1], g.hf[2], g.hf[3], g.hf[4], g.hf[5], g.hf[6], g.hf[7], g.hf[8]};
    auto test = [&](int j, int tj, int Sa, int Sb, int Sc, float4 pj4) {
        if (j == (int)i && Sa == 0 && Sb == 0 && Sc == 0) return;
        const float fa = (float)Sa, fb = (float)Sb, fc = (float)Sc;
        float q[3], B[3];
        const float pjv[3] = {pj4.x, pj4.y, pj4.z};
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const float ta = __fmul_rn(fa, hf[x]), tb = __fmul_rn(fb, hf[3 + x]), tc = __fmul_rn(fc, hf[6 + x]);
            q[x] = __fadd_rn(__fsub_rn(pjv[x], pi[x]), __fadd_rn(__fadd_rn(ta, tb), tc));
            B[x] = fabsf(pjv[x]) + fabsf(pi[x]) + fabsf(ta) + fabsf(tb) + fabsf(tc);
        }
        const float r2q = __fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])), __fmul_rn(q[2], q[2]));
        if (r2q > rcq2) return;
        if (Sa < -SMAX || Sa > SMAX || Sb < -SMAX || Sb > SMAX || Sc < -SMAX || Sc > SMAX) {
            atomic_err(err, 2);
            return;
        }
        constexpr float EPS = 9.5367431640625e-07f;  // 2^-20
        float M = EPS * r2q;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const float dx = EPS * B[x];
            M += 2.0f * fabsf(q[x]) * dx + dx * dx;
        }
        const float lo = r2q - M, hi = r2q + M;
        bool inR, inA;
        if ((hi < rc2R || lo >= rc2R) && (hi < rc2A || lo >= rc2A)) {
            inR = hi < rc2R;
            inA = hi < rc2A;
        } else {  // within the error band of a cutoff: the exact predicate
            float d32[3];
            const float r2 = pair_d(pi, pos + 3 * j, g.h, Sa, Sb, Sc, d32);
            inR = r2 < rc2R;
            inA = r2 < rc2A;
        }
        if (inR) hit(j, tj, Sa, Sb, Sc, inA);
    };
    if (g.n[0] == 1 && g.n[1] == 1 && g.n[2] == 1) {
        // Image box of each candidate j in FP32, widened by more than the FP32 rounding of
        // f = (p_j - p_i) h^-1 (relative 2^-20 of the magnitudes involved), so it holds every
        // image the exact box holds; the extra images are rejected by the pair predicate.
        // Only a box that reaches past the packed shift range is recomputed in FP64.
        const float *invf = g.invf;
        for (int64_t j = atom_off[s] + lane; j < atom_off[s + 1]; j += 32) {
            const float4 pj = pos4[j];
            const float d0[3] = {pj.x - pi[0], pj.y - pi[1], pj.z - pi[2]};
            int lo[3], hi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float R = rcq * g.nb[a];
                const float f = d0[0] * invf[a] + d0[1] * invf[3 + a] + d0[2] * invf[6 + a];
                const float bound = fabsf(d0[0] * invf[a]) + fabsf(d0[1] * invf[3 + a]) + fabsf(d0[2] * invf[6 + a]);
                const float m = 0x1p-20f * (bound + R) + 1e-30f;
                lo[a] = (int)ceilf(-f - R - m);
                hi[a] = (int)floorf(-f + R + m);
                if (lo[a] < -SMAX - 1 || hi[a] > SMAX + 1) {
                    const double fd = ((double)pj.x - (double)pi[0]) * g.inv[a] +
                                      ((double)pj.y - (double)pi[1]) * g.inv[3 + a] +
                                      ((double)pj.z - (double)pi[2]) * g.inv[6 + a];
                    const double Rd = (double)rcq * sqrt(g.inv[a] * g.inv[a] + g.inv[3 + a] * g.inv[3 + a] +
                                                         g.inv[6 + a] * g.inv[6 + a]);
                    lo[a] = (int)ceil(-fd - Rd);
                    hi[a] = (int)floor(-fd + Rd);
                }
                if (lo[a] < -SMAX - 1 || hi[a] > SMAX + 1) {  // beyond the packed shift range
                    atomic_err(err, 2);
                    lo[a] = 1;
                    hi[a] = 0;
                }
            }
            for (int Sa = lo[0]; Sa <= hi[0]; ++Sa)
                for (int Sb = lo[1]; Sb <= hi[1]; ++Sb)
                    for (int Sc = lo[2]; Sc <= hi[2]; ++Sc) test((int)j, __float_as_int(pj.w), Sa, Sb, Sc, pj);
        }
        return;
    }
    const int64_t lb = atom_bin[i] - bin_off[s];
    const int bi[3] = {(int)(lb / ((int64_t)g.n[1] * g.n[2])), (int)((lb / g.n[2]) % g.n[1]), (int)(lb % g.n[2])};
    const int4 wi = atom_wrap[i];
    for (int da = -g.m[0]; da <= g.m[0]; ++da) {
        int ba = bi[0] + da;
        const int sa = (ba >= 0) ? ba / g.n[0] : -((-ba + g.n[0] - 1) / g.n[0]);
        ba -= sa * g.n[0];
        for (int db = -g.m[1]; db <= g.m[1]; ++db) {
            int bb = bi[1] + db;
            const int sb = (bb >= 0) ? bb / g.n[1] : -((-bb + g.n[1] - 1) / g.n[1]);
            bb -= sb * g.n[1];
            // the bins along c in runs of consecutive bins with one shift: their atoms are
            // consecutive in bin order, so the lanes take each run as one range
            for (int dc = -g.m[2]; dc <= g.m[2];) {
                int bc = bi[2] + dc;
                const int sc = (bc >= 0) ? bc / g.n[2] : -((-bc + g.n[2] - 1) / g.n[2]);
                bc -= sc * g.n[2];
                const int run = min(g.m[2] - dc, g.n[2] - 1 - bc);  // further bins in this run
                const int64_t bin = bin_off[s] + ((int64_t)ba * g.n[1] + bb) * g.n[2] + bc;
                for (int64_t t = bin_start[bin] + lane; t < bin_start[bin + run + 1]; t += 32) {
                    const float4 bp = bin_pos[t];  // the bins' atoms in bin order: coalesced
                    const int4 wj = bin_wrap[t];
                    const int jt = __float_as_int(bp.w);
                    test(jt >> 4, jt & 15, sa + wi.x - wj.x, sb + wi.y - wj.y, sc + wi.z - wj.z, bp);
                }
                dc += run + 1;
            }
        }
    }
}

__device__ __forceinline__ uint64_t pair_key(bool ang, int tj, int j, int Sa, int Sb, int Sc) {
    const uint64_t grp = ang ? 0ull : 1ull;  // angular neighbours first
    return (grp << 63) | ((uint64_t)tj << 59) | ((uint64_t)j << 24) | (uint64_t)pack_shift(Sa, Sb, Sc);
}

// Pair counts per atom (one warp per atom), and the sort keys of the first `cap` pairs
// of each atom in scratch[i * cap ...] (unordered): when no atom has more, the keys need
// no second scan.  *overflow is set when some atom has more than cap pairs.
__global__ void __launch_bounds__(256, 4) k_count_w(int64_t na, const float *pos, const float4 *pos4, const int *struct_of,
                          const int64_t *atom_off, const SGeom *geom, const int64_t *bin_off, const int64_t *atom_bin,
                          const int4 *atom_wrap, const int64_t *bin_start, const float4 *bin_pos,
                          const int4 *bin_wrap, float rc2R,
                          float rc2A, float rcq, int64_t *cnt, int *n_ang, uint64_t *scratch, int cap, int *overflow,
                          int *err) {
    __shared__ int slot[32];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (i >= na) return;
    if (lane == 0) slot[wib] = 0;
    __syncwarp();
    int nang = 0;
    uint64_t *dst = scratch + i * (int64_t)cap;
    scan_atom_warp(i, lane, pos, pos4, struct_of, atom_off, geom, bin_off, atom_bin, atom_wrap, bin_start, bin_pos, bin_wrap,
                   rc2R, rc2A, rcq * rcq, rcq, err, [&](int j, int tj, int Sa, int Sb, int Sc, bool ang) {
                       const int k = atomicAdd(&slot[wib], 1);
                       if (k < cap) dst[k] = pair_key(ang, tj, j, Sa, Sb, Sc);
                       if (ang) ++nang;
                   });
    nang = __reduce_add_sync(FULL, nang);
    __syncwarp();
    if (lane == 0) {
        const int nr = slot[wib];
        cnt[i] = nr;
        n_ang[i] = nang;
        if (nr > cap) atomicOr(overflow, 1);
    }
}

// Sort keys of every pair (one warp per atom); slots taken through a shared counter.
__global__ void k_fill_w(int64_t na, const float *pos, const float4 *pos4, const int *struct_of,
                         const int64_t *atom_off,
                         const SGeom *geom, const int64_t *bin_off, const int64_t *atom_bin, const int4 *atom_wrap,
                         const int64_t *bin_start, const float4 *bin_pos, const int4 *bin_wrap, float rc2R,
                         float rc2A, float rcq,
                         const int64_t *nbr_off, uint64_t *keys, int *err) {
    __shared__ int slot[32];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (i >= na) return;
    if (lane == 0) slot[wib] = 0;
    __syncwarp();
    const int64_t o = nbr_off[i], n = nbr_off[i + 1] - o;
    scan_atom_warp(i, lane, pos, pos4, struct_of, atom_off, geom, bin_off, atom_bin, atom_wrap, bin_start, bin_pos, bin_wrap,
                   rc2R, rc2A, rcq * rcq, rcq, err, [&](int j, int tj, int Sa, int Sb, int Sc, bool ang) {
                       const int k = atomicAdd(&slot[wib], 1);
                       if (k < n) keys[o + k] = pair_key(ang, tj, j, Sa, Sb, Sc);
                   });
    __syncwarp();
    if (lane == 0 && slot[wib] != n) atomic_err(err, 5);
}

constexpr uint32_t SHIFT0 = 0x808080u;  // packed S = (0, 0, 0)

// Stores key k at its sorted position with its pair record (displacement, j and its species).
__device__ __forceinline__ void store_pair(uint64_t k, int64_t slot, const float *d32, uint64_t *keys_out,
                                           float4 *pair, int32_t *shift) {
    keys_out[slot] = k;
    const int j = (int)((k >> 24) & ((1ull << 35) - 1));
    const int tj = (int)((k >> 59) & 15ull);
    pair[slot] = make_float4(d32[0], d32[1], d32[2], __int_as_float((j << 4) | tj));
    shift[slot] = (int32_t)(k & 0xffffffull);
}

// pair_d's displacement for a pair with S = (0, 0, 0), in FP32 and with the same bits.
// p_j - p_i of two floats is exact in FP64 unless one operand is below 2^-29 of the other,
// and then both fl32(p_j - p_i) and fl32(fl64(p_j - p_i)) are the larger operand.  The
// image term 0 h_a + 0 h_b + 0 h_c is a signed zero (negative only when all three h
// components are), and adding it follows the same sign rules in either precision.
__device__ __forceinline__ void pair_d0(const float *pi, const float *pj, const double *h, float *d32) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const bool neg = (__double_as_longlong(h[x]) & __double_as_longlong(h[3 + x]) &
                          __double_as_longlong(h[6 + x])) < 0;
        d32[x] = __fadd_rn(__fsub_rn(pj[x], pi[x]), neg ? -0.0f : 0.0f);
    }
}

// The predicate's float displacement of the pair of key k from atom i.
__device__ __forceinline__ void decode_key(uint64_t k, int64_t i, const float *pos, const SGeom &g, float *d32) {
    const int j = (int)((k >> 24) & ((1ull << 35) - 1));
    const uint32_t sp = (uint32_t)(k & 0xffffffull);
    if (sp == SHIFT0) {
        pair_d0(pos + 3 * i, pos + 3 * j, g.h, d32);
    } else {
        const int Sa = (int)((sp >> 16) & 255) - 128, Sb = (int)((sp >> 8) & 255) - 128, Sc = (int)(sp & 255) - 128;
        if (!pair_d_fp32(pos + 3 * i, pos + 3 * j, g.hf, Sa, Sb, Sc, d32))
            pair_d(pos + 3 * i, pos + 3 * j, g.h, Sa, Sb, Sc, d32);
    }
}

// Pair record of key k from the predicate's displacement.
__device__ __forceinline__ void emit_pair(uint64_t k, int64_t slot, int64_t i, const float *pos, const SGeom &g,
                                          uint64_t *keys_out, float4 *pair, int32_t *shift) {
    float d32[3];
    decode_key(k, i, pos, g, d32);
    store_pair(k, slot, d32, keys_out, pair, shift);
}

// Rank sort of n <= 32 R staged keys: lane l owns keys l, l + 32, ...; every staged key
// is read once per lane, two at a time (a 16-byte broadcast), against the owned keys in
// registers.  sk holds n keys padded to an even count with a key above all others.
// Pairs with S = 0 are then written at once (FP32); the others are queued in sk / sq and
// written by consecutive lanes, so that the FP64 displacements run on full warps.
template <int R>
__device__ __forceinline__ void rank_staged(uint64_t *sk, int *sq, int n, int lane, int64_t beg, int64_t i,
                                            const float *pos, const SGeom &g, uint64_t *keys_out, float4 *pair,
                                            int32_t *shift) {
    uint64_t own[R];
    int rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane + 32 * r;
        own[r] = e < n ? sk[e] : 0ull;
        rank[r] = 0;
    }
    const ulonglong2 *sk2 = reinterpret_cast<const ulonglong2 *>(sk);
    for (int e2 = 0; e2 < (n + 1) >> 1; ++e2) {
        const ulonglong2 kk = sk2[e2];
#pragma unroll
        for (int r = 0; r < R; ++r) rank[r] += (kk.x < own[r] ? 1 : 0) + (kk.y < own[r] ? 1 : 0);
    }
    __syncwarp();  // every lane has read the staged keys: sk / sq now take the queue
    int nq = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool valid = lane + 32 * r < n;
        const bool img = valid && (uint32_t)(own[r] & 0xffffffull) != SHIFT0;
        const unsigned m = __ballot_sync(FULL, img);
        if (img) {
            const int q = nq + __popc(m & ((1u << lane) - 1u));
            sk[q] = own[r];
            sq[q] = rank[r];
        } else if (valid) {
            const int j = (int)((own[r] >> 24) & ((1ull << 35) - 1));
            float d32[3];
            pair_d0(pos + 3 * i, pos + 3 * j, g.h, d32);
            store_pair(own[r], beg + rank[r], d32, keys_out, pair, shift);
        }
        nq += __popc(m);
    }
    __syncwarp();
    for (int q = lane; q < nq; q += 32) emit_pair(sk[q], beg + sq[q], i, pos, g, keys_out, pair, shift);
}

// One warp per atom: the atom's keys in ascending order (angular flag, species of j, j, S)
// with their pair records (displacement = the predicate's pair_d, j and its species).
__global__ void k_sort_decode(int64_t na, const uint64_t *keys_in, const uint64_t *scratch, int cap,
                              const int64_t *nbr_off, const float *pos,
                              const int *struct_of, const SGeom *geom, uint64_t *keys_out, float4 *pair,
                              int32_t *shift) {
    constexpr int STAGE = 256;  // keys per warp staged in shared memory
    __shared__ __align__(16) uint64_t sk[8][STAGE];
    __shared__ int sq[8][STAGE];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (i >= na) return;
    const int64_t beg = nbr_off[i], n = nbr_off[i + 1] - beg;
    const SGeom &g = geom[struct_of[i]];
    const uint64_t *src = scratch ? scratch + i * (int64_t)cap : keys_in + beg;
    if (n <= STAGE) {
        uint64_t *s = sk[wib];
        for (int64_t e = lane; e < n; e += 32) s[e] = src[e];
        if (lane == 0 && (n & 1)) s[n] = ~0ull;  // n odd: n < STAGE, pad above every key
        __syncwarp();
        const int nn = (int)n;
        int *q = sq[wib];
        switch ((nn + 31) >> 5) {
            case 0: break;
            case 1: rank_staged<1>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 2: rank_staged<2>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 3: rank_staged<3>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 4: rank_staged<4>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 5: rank_staged<5>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 6: rank_staged<6>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            case 7: rank_staged<7>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
            default: rank_staged<8>(s, q, nn, lane, beg, i, pos, g, keys_out, pair, shift); break;
        }
        return;
    }
    // longer lists: rank against the keys in global memory
    for (int64_t e = lane; e < n; e += 32) {
        const uint64_t k = src[e];
        int64_t rank = 0;
        for (int64_t e2 = 0; e2 < n; ++e2) rank += (src[e2] < k) ? 1 : 0;
        emit_pair(k, beg + rank, i, pos, g, keys_out, pair, shift);
    }
}

// Reverse-pair index, one thread per pair (the lanes of a warp over one atom's list).  Each
// unordered pair {(i, j, S), (j, i, -S)} is searched once, from the entry with i < j (or,
// for an atom's own images, the larger packed shift): a binary search of j's sorted keys,
// then rev set on both entries and the displacements checked for antisymmetry.  Every found pair adds one to *found; the host checks 2 found == M, so an
// entry without a partner cannot pass unnoticed.
__global__ void k_reverse(int64_t na, const int64_t *nbr_off, const uint64_t *keys, const int *type, int *rev,
                          const float4 *pair, unsigned long long *found, int *err) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= na) return;
    const int64_t beg = nbr_off[i], end = nbr_off[i + 1];
    const int ti = type[i];
    unsigned nf = 0;
    for (int64_t p = beg + lane; p < end; p += 32) {
        const uint64_t k = keys[p];
        const int j = (int)((k >> 24) & ((1ull << 35) - 1));
        const uint32_t sp = (uint32_t)(k & 0xffffffull);
        const int Sa = (int)((sp >> 16) & 255) - 128, Sb = (int)((sp >> 8) & 255) - 128, Sc = (int)(sp & 255) - 128;
        const uint32_t spn = pack_shift(-Sa, -Sb, -Sc);
        if (!(j > (int)i || (j == (int)i && sp > spn))) continue;  // the partner's entry searches
        const uint64_t want = (k & (1ull << 63)) | ((uint64_t)ti << 59) | ((uint64_t)i << 24) | (uint64_t)spn;
        int64_t lo = nbr_off[j], hi = nbr_off[j + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= nbr_off[j + 1] || keys[lo] != want) {
            atomic_err(err, 6);
            continue;
        }
        rev[p] = (int)lo;
        rev[lo] = (int)p;
        ++nf;
        if (pair) {  // candidate lists carry no records
            const float4 a = pair[p], b = pair[lo];
            if (a.x != -b.x || a.y != -b.y || a.z != -b.z) atomic_err(err, 7);
        }
    }
    nf = __reduce_add_sync(FULL, nf);
    if (lane == 0 && nf) atomicAdd(found, (unsigned long long)nf);
}

// Candidate keys of each atom in ascending order (one warp per atom, rank sort).
__global__ void k_sort_keys(int64_t na, const uint64_t *keys_in, const uint64_t *scratch, int cap,
                            const int64_t *off, uint64_t *keys_out) {
    constexpr int STAGE = 256;  // keys per warp staged in shared memory
    __shared__ __align__(16) uint64_t sk[8][STAGE];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (i >= na) return;
    const int64_t beg = off[i], n = off[i + 1] - beg;
    const uint64_t *src = scratch ? scratch + i * (int64_t)cap : keys_in + beg;
    if (n <= STAGE) {
        uint64_t *s = sk[wib];
        for (int64_t e = lane; e < n; e += 32) s[e] = src[e];
        __syncwarp();
        for (int64_t e = lane; e < n; e += 32) {
            const uint64_t k = s[e];
            int rank = 0;
            for (int e2 = 0; e2 < (int)n; ++e2) rank += s[e2] < k ? 1 : 0;
            keys_out[beg + rank] = k;
        }
        return;
    }
    for (int64_t e = lane; e < n; e += 32) {
        const uint64_t k = src[e];
        int64_t rank = 0;
        for (int64_t e2 = 0; e2 < n; ++e2) rank += (src[e2] < k) ? 1 : 0;
        keys_out[beg + rank] = k;
    }
}

// max_i |p_i - r_i|^2 in FP64 (as the bits of a non-negative double: integer order).
__global__ void k_max_disp(int64_t na, const float *pos, const float *ref, unsigned long long *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (i < na) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const double d = (double)pos[3 * i + x] - (double)ref[3 * i + x];
            d2 += d * d;
        }
        if (!(d2 <= 1e30)) d2 = 1e30;  // a non-finite position: the scan rejects it
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(d2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, b, o);
        b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

// Candidate filter, one warp per atom.  Pass 1 (WRITE = false): the pair predicate (above) of
// every candidate at the current positions, as flags (bit 0 within r_c^R, bit 1 within
// r_c^A) and its pair record in crec, and the atom's radial and angular counts.  Pass 2:
// the kept candidates' records at their list positions (angular ones first, each group in
// candidate order) and each candidate's position (pidx, -1 if dropped).
template <bool WRITE>
__global__ void k_filter(int64_t na, const int64_t *coff, const uint64_t *ckey, const float *pos,
                         const int *struct_of, const SGeom *geom, float rc2R, float rc2A, uint8_t *cflag,
                         float4 *crec, int64_t *cnt, int *n_ang, const int64_t *nbr_off, float4 *pair,
                         int32_t *shift, int *pidx) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= na) return;
    const int64_t beg = coff[i], n = coff[i + 1] - beg;
    const SGeom &g = geom[struct_of[i]];
    if (!WRITE) {
        int nr = 0, nang = 0;
        for (int64_t e = lane; e < n; e += 32) {
            const uint64_t k = ckey[beg + e];
            float d32[3];
            decode_key(k, i, pos, g, d32);
            const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(d32[0], d32[0]), __fmul_rn(d32[1], d32[1])),
                                       __fmul_rn(d32[2], d32[2]));
            const bool inR = r2 < rc2R, inA = r2 < rc2A;
            cflag[beg + e] = (uint8_t)((inR ? 1 : 0) | (inA ? 2 : 0));
            if (inR) {
                const int j = (int)((k >> 24) & ((1ull << 35) - 1));
                const int tj = (int)((k >> 59) & 15ull);
                crec[beg + e] = make_float4(d32[0], d32[1], d32[2], __int_as_float((j << 4) | tj));
            }
            nr += inR ? 1 : 0;
            nang += inA ? 1 : 0;
        }
        nr = __reduce_add_sync(FULL, nr);
        nang = __reduce_add_sync(FULL, nang);
        if (lane == 0) {
            cnt[i] = nr;
            n_ang[i] = nang;
        }
        return;
    }
    const int64_t pbeg = nbr_off[i];
    const int nA = n_ang[i];
    int ca = 0, cr = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t e0 = 0; e0 < n; e0 += 32) {
        const int64_t e = e0 + lane;
        const int f = e < n ? cflag[beg + e] : 0;
        const bool isA = (f & 2) != 0, isR = (f & 1) != 0 && !isA;
        const unsigned mA = __ballot_sync(FULL, isA), mR = __ballot_sync(FULL, isR);
        int64_t slot = -1;
        if (isA) slot = pbeg + ca + __popc(mA & below);
        else if (isR) slot = pbeg + nA + cr + __popc(mR & below);
        if (slot >= 0) {
            pair[slot] = crec[beg + e];
            shift[slot] = (int32_t)(ckey[beg + e] & 0xffffffull);
        }
        if (e < n) pidx[beg + e] = (int)slot;
        ca += __popc(mA);
        cr += __popc(mR);
    }
}

// rev of the filtered lists from the candidates' reverse index.
__global__ void k_filter_rev(int64_t Mc, const int *pidx, const int *crev, int *rev) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Mc) return;
    const int p = pidx[q];
    if (p >= 0) rev[p] = pidx[crev[q]];
}

// out += sum of v[0..n) (integer atomics: the total does not depend on the order)
__global__ void k_sum_int(int64_t n, const int *v, int64_t *out) {
    long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0) atomicAdd((unsigned long long *)out, (unsigned long long)s);
}

}  // namespace

namespace {

// Per-structure bin grids for a cutoff rc (they depend on the cells only).
struct Grid {
    DevBuf *geom, *nbins, *bin_off;
    int64_t *nbin_total;
    bool *ok;
};

int grid_setup(Ctx *c, const Grid &gr, float rc, bool same_cells, bool with_struct_of) {
    const int64_t ns = c->n_struct;
    const cudaStream_t st = c->stream;
    int *err = c->d_err.as<int>();
    if (gr.geom->ensure_bytes(sizeof(SGeom) * (size_t)(ns > 0 ? ns : 1)) || gr.nbins->ensure<int64_t>(ns + 1) ||
        gr.bin_off->ensure<int64_t>(ns + 1) || c->d_total.ensure<int64_t>(8))
        return c->fail(NEP_ENOMEM, "geometry buffers");
    if (same_cells && *gr.ok) return NEP_OK;
    *gr.ok = false;
    if (ns > 0) {
        k_struct_geom<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(ns, c->cell.as<float>(), (double)rc,
                                                                    (SGeom *)gr.geom->ptr, gr.nbins->as<int64_t>(), err);
        if (with_struct_of)
            k_struct_of<<<(unsigned)ns, 128, 0, st>>>(ns, c->atom_off.as<int64_t>(), c->struct_of.as<int>());
    }
    CK(cudaGetLastError());
    int rc_ = scan_exclusive(c, gr.nbins->as<int64_t>(), ns, gr.bin_off->as<int64_t>(), c->d_total.as<int64_t>());
    if (rc_) return rc_;
    int64_t nbt = 0;
    int herr = 0;
    CK(cudaMemcpyAsync(&nbt, c->d_total.as<int64_t>(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return c->fail(NEP_EINVAL, herr == 1 ? "singular or non-finite cell" : "cell too thin for the cutoff (more than 127 images)");
    *gr.nbin_total = nbt;
    *gr.ok = true;
    return NEP_OK;
}

// Binning and the counting scan at cutoffs (rcR, rcA) over grid gr: the pair counts of the
// atoms scanned into off [na + 1] (total M), the first `cap` keys of each atom in
// nbr_scratch, the angular counts in n_ang, and whether some atom has more than cap pairs.
int scan_count(Ctx *c, const Grid &gr, float rcR, float rcA, int cap, DevBuf &off, int64_t &M, int &overflow) {
    const int64_t na = c->n_atoms;
    const cudaStream_t st = c->stream;
    const float rc2R = rcR * rcR, rc2A = rcA * rcA;  // single rounded products
    const float rcq = rcR + 0.05f;
    int *err = c->d_err.as<int>();
    const SGeom *geom = (const SGeom *)gr.geom->ptr;
    const int64_t nbin_total = *gr.nbin_total;
    if (c->bin_cnt.ensure<int64_t>(nbin_total + 1) || c->bin_start.ensure<int64_t>(nbin_total + 1) ||
        c->bin_cur.ensure<int64_t>(nbin_total + 1) || c->atom_bin.ensure<int64_t>(na + 1) ||
        c->atom_wrap.ensure_bytes(sizeof(int4) * (size_t)(na + 1)) || c->bin_atoms.ensure<int>(na + 1) ||
        c->cnt.ensure<int64_t>(na + 1) || c->n_ang.ensure<int>(na + 1) || off.ensure<int64_t>(na + 1) ||
        c->pos4.ensure<float4>(na + 1) || c->d_flag.ensure<int>(1) || c->bin_pos.ensure<float4>(na + 1) ||
        c->bin_wrap.ensure_bytes(sizeof(int4) * (size_t)(na + 1)) ||
        c->nbr_scratch.ensure<uint64_t>(na * (int64_t)cap + 1))
        return c->fail(NEP_ENOMEM, "bin buffers");
    CK(cudaMemsetAsync(c->d_flag.ptr, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c->bin_cnt.ptr, 0, sizeof(int64_t) * (size_t)(nbin_total + 1), st));
    CK(cudaMemsetAsync(c->bin_cur.ptr, 0, sizeof(int64_t) * (size_t)(nbin_total + 1), st));
    const unsigned gA = (unsigned)((na + 255) / 256);     // 256-thread blocks, one thread per atom
    const unsigned gW = (unsigned)((na * 32 + 255) / 256);  // 256-thread blocks, one warp per atom
    CK(cudaMemsetAsync(c->cnt.ptr, 0, sizeof(int64_t) * (size_t)(na + 1), st));
    CK(cudaMemsetAsync(c->n_ang.ptr, 0, sizeof(int) * (size_t)(na + 1), st));
    if (na > 0) {
        k_atom_bin<<<gA, 256, 0, st>>>(na, c->pos.as<float>(), c->type.as<int>(), c->cfg.n_types,
                                       c->struct_of.as<int>(), geom, gr.bin_off->as<int64_t>(),
                                       c->atom_bin.as<int64_t>(), (int4 *)c->atom_wrap.ptr, c->bin_cnt.as<int64_t>(),
                                       c->pos4.as<float4>(), err);
        CK(cudaGetLastError());
    }
    int rc = scan_exclusive(c, c->bin_cnt.as<int64_t>(), nbin_total, c->bin_start.as<int64_t>(),
                            c->d_total.as<int64_t>() + 1);
    if (rc) return rc;
    if (na > 0) {
        k_bin_fill<<<gA, 256, 0, st>>>(na, c->atom_bin.as<int64_t>(), c->bin_start.as<int64_t>(),
                                       c->bin_cur.as<int64_t>(), c->bin_atoms.as<int>());
        k_bin_pack<<<gA, 256, 0, st>>>(na, c->bin_atoms.as<int>(), c->pos4.as<float4>(),
                                       (const int4 *)c->atom_wrap.ptr, c->bin_pos.as<float4>(),
                                       (int4 *)c->bin_wrap.ptr);
        k_count_w<<<gW, 256, 0, st>>>(na, c->pos.as<float>(), c->pos4.as<float4>(),
                                      c->struct_of.as<int>(), c->atom_off.as<int64_t>(), geom,
                                      gr.bin_off->as<int64_t>(), c->atom_bin.as<int64_t>(),
                                      (const int4 *)c->atom_wrap.ptr, c->bin_start.as<int64_t>(),
                                      c->bin_pos.as<float4>(), (const int4 *)c->bin_wrap.ptr, rc2R, rc2A, rcq,
                                      c->cnt.as<int64_t>(),
                                      c->n_ang.as<int>(), c->nbr_scratch.as<uint64_t>(), cap, c->d_flag.as<int>(), err);
        CK(cudaGetLastError());
    }
    rc = scan_exclusive(c, c->cnt.as<int64_t>(), na, off.as<int64_t>(), c->d_total.as<int64_t>());
    if (rc) return rc;
    int herr = 0;
    M = 0;
    overflow = 0;
    CK(cudaMemcpyAsync(&M, c->d_total.as<int64_t>(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&overflow, c->d_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return c->fail(NEP_EINVAL, herr == 3 ? "species index out of range" :
                                          herr == 4 ? "non-finite or far out-of-cell position" :
                                                      "more than 127 periodic images along a cell vector");
    if (M >= (int64_t)1 << 31) return c->fail(NEP_EINVAL, "more than 2^31 neighbour pairs");
    return NEP_OK;
}

// the second scan of the keys when some atom has more than cap pairs
void fill_keys(Ctx *c, const Grid &gr, float rcR, float rcA, const DevBuf &off, uint64_t *keys) {
    const int64_t na = c->n_atoms;
    const unsigned gW = (unsigned)((na * 32 + 255) / 256);
    k_fill_w<<<gW, 256, 0, c->stream>>>(na, c->pos.as<float>(), c->pos4.as<float4>(), c->struct_of.as<int>(),
                                        c->atom_off.as<int64_t>(), (const SGeom *)gr.geom->ptr,
                                        gr.bin_off->as<int64_t>(), c->atom_bin.as<int64_t>(),
                                        (const int4 *)c->atom_wrap.ptr, c->bin_start.as<int64_t>(),
                                        c->bin_pos.as<float4>(), (const int4 *)c->bin_wrap.ptr, rcR * rcR, rcA * rcA,
                                        rcR + 0.05f, off.as<int64_t>(), keys, c->d_err.as<int>());
}

int key_cap(int64_t na) { return (int)std::min<int64_t>(128, (int64_t)8e9 / (8 * std::max<int64_t>(na, 1))); }

}  // namespace

int build_neighbors(Ctx *c, bool same_cells, bool host_lists) {
    const int64_t na = c->n_atoms;
    const cudaStream_t st = c->stream;
    const float rcR = c->cfg.rc_R, rcA = c->cfg.rc_A;
    int *err = c->d_err.as<int>();
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (!same_cells) c->cand_ok = c->cgeom_ok = false;  // candidates hold the old cells
    const Grid gr{&c->geom, &c->nbins, &c->bin_off, &c->nbin_total, &c->geom_ok};
    int rc = grid_setup(c, gr, rcR, same_cells, true);
    if (rc) return rc;
    // keys of up to `cap` pairs per atom are kept from the counting scan (at most 8 GB)
    const int cap = key_cap(na);
    int64_t M = 0;
    int overflow = 0;
    if ((rc = scan_count(c, gr, rcR, rcA, cap, c->nbr_off, M, overflow))) return rc;
    if ((overflow && c->keys_tmp.ensure<uint64_t>(M + 1)) || c->keys.ensure<uint64_t>(M + 1) ||
        c->pair.ensure_bytes(sizeof(float4) * (size_t)(M + 1)) || c->rev.ensure<int>(M + 1) ||
        c->shift.ensure<int32_t>(M + 1))
        return c->fail(NEP_ENOMEM, "pair buffers");
    c->n_pairs = M;
    const SGeom *geom = (const SGeom *)c->geom.ptr;
    const unsigned gw = (unsigned)((na * 32 + 255) / 256);
    if (na > 0) {
        if (overflow) fill_keys(c, gr, rcR, rcA, c->nbr_off, c->keys_tmp.as<uint64_t>());
        k_sort_decode<<<gw, 256, 0, st>>>(na, c->keys_tmp.as<uint64_t>(),
                                          overflow ? nullptr : c->nbr_scratch.as<uint64_t>(), cap,
                                          c->nbr_off.as<int64_t>(),
                                          c->pos.as<float>(), c->struct_of.as<int>(), geom, c->keys.as<uint64_t>(),
                                          (float4 *)c->pair.ptr, c->shift.as<int32_t>());
    }
    // found reverse pairs and the angular pair count (integer sums: exact in any order)
    int64_t *found_dev = c->d_total.as<int64_t>() + 4;
    int64_t *nang_dev = c->d_total.as<int64_t>() + 5;
    CK(cudaMemsetAsync(found_dev, 0, 2 * sizeof(int64_t), st));
    if (na > 0) {
        k_reverse<<<gw, 256, 0, st>>>(na, c->nbr_off.as<int64_t>(), c->keys.as<uint64_t>(), c->type.as<int>(),
                                      c->rev.as<int>(), (const float4 *)c->pair.ptr,
                                      (unsigned long long *)found_dev, err);
        CK(cudaGetLastError());
    }
    if (na > 0) k_sum_int<<<(unsigned)std::min<int64_t>((na + 255) / 256, 1024), 256, 0, st>>>(na, c->n_ang.as<int>(), nang_dev);
    CK(cudaGetLastError());
    int64_t fin[2] = {0, 0};  // found reverse pairs, angular pairs
    int herr = 0;
    CK(cudaMemcpyAsync(fin, found_dev, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr || 2 * fin[0] != M) return c->fail(NEP_EINTERNAL, "neighbour list is not symmetric");
    c->n_pairs_ang = fin[1];
    c->h_lists_ok = false;
    return host_lists ? fetch_host_lists(c) : NEP_OK;
}

// ----------------------------------------------------------------------------- candidate lists
// Position updates with the cells kept.  A candidate list holds, for reference positions R,
// every pair within r_c + s (s the skin).  If no atom has moved more than d from R, a pair
// within r_c at the new positions was within r_c + 2d at R, so for 2d < s the new lists are
// the candidates that pass the pair predicate at the new positions: a filter instead
// of a scan.  The filter keeps the candidates' order, (t_j, j, S), and puts the angular
// ones first, which is the order the scan's sort gives: the lists are the scan's, bit for
// bit.  The reverse index follows from the candidates' own.

int build_candidates(Ctx *c) {
    const int64_t na = c->n_atoms;
    const cudaStream_t st = c->stream;
    const float rcc = c->cfg.rc_R + c->skin;
    int *err = c->d_err.as<int>();
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    c->cand_ok = false;
    const Grid gr{&c->cgeom, &c->cnbins, &c->cbin_off, &c->cnbin_total, &c->cgeom_ok};
    int rc = grid_setup(c, gr, rcc, true, false);
    if (rc) return rc;
    const int cap = key_cap(na);
    int64_t Mc = 0;
    int overflow = 0;
    if ((rc = scan_count(c, gr, rcc, rcc, cap, c->cand_off, Mc, overflow))) return rc;
    // the lists the filter writes are at most the candidates: room for them once
    if ((overflow && c->keys_tmp.ensure<uint64_t>(Mc + 1)) || c->cand_key.ensure<uint64_t>(Mc + 1) ||
        c->cand_rev.ensure<int>(Mc + 1) || c->cand_pidx.ensure<int>(Mc + 1) || c->cand_flag.ensure<uint8_t>(Mc + 1) ||
        c->cand_rec.ensure_bytes(sizeof(float4) * (size_t)(Mc + 1)) ||
        c->cand_ref.ensure<float>(3 * na + 1) || c->pair.ensure_bytes(sizeof(float4) * (size_t)(Mc + 1)) ||
        c->rev.ensure<int>(Mc + 1) || c->shift.ensure<int32_t>(Mc + 1) ||
        c->G.ensure_bytes(sizeof(float4) * (size_t)(Mc + 1)))
        return c->fail(NEP_ENOMEM, "candidate buffers");
    int64_t *found_dev = c->d_total.as<int64_t>() + 4;
    CK(cudaMemsetAsync(found_dev, 0, sizeof(int64_t), st));
    if (na > 0) {
        const unsigned gw = (unsigned)((na * 32 + 255) / 256);
        if (overflow) fill_keys(c, gr, rcc, rcc, c->cand_off, c->keys_tmp.as<uint64_t>());
        k_sort_keys<<<gw, 256, 0, st>>>(na, c->keys_tmp.as<uint64_t>(),
                                        overflow ? nullptr : c->nbr_scratch.as<uint64_t>(), cap,
                                        c->cand_off.as<int64_t>(), c->cand_key.as<uint64_t>());
        k_reverse<<<gw, 256, 0, st>>>(na, c->cand_off.as<int64_t>(), c->cand_key.as<uint64_t>(), c->type.as<int>(),
                                      c->cand_rev.as<int>(), nullptr, (unsigned long long *)found_dev, err);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(c->cand_ref.ptr, c->pos.ptr, sizeof(float) * 3 * na, cudaMemcpyDeviceToDevice, st));
    }
    int64_t found = 0;
    int herr = 0;
    CK(cudaMemcpyAsync(&found, found_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr || 2 * found != Mc) return c->fail(NEP_EINTERNAL, "candidate list is not symmetric");
    c->cand_M = Mc;
    c->cand_ok = true;
    return NEP_OK;
}

int filter_candidates(Ctx *c, bool host_lists, bool &moved_too_far) {
    const int64_t na = c->n_atoms, Mc = c->cand_M;
    const cudaStream_t st = c->stream;
    const float rcR = c->cfg.rc_R, rcA = c->cfg.rc_A;
    int *err = c->d_err.as<int>();
    moved_too_far = false;
    CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    int64_t *disp_dev = c->d_total.as<int64_t>() + 6;  // max squared displacement (FP64 bits)
    int64_t *nang_dev = c->d_total.as<int64_t>() + 5;
    CK(cudaMemsetAsync(nang_dev, 0, 2 * sizeof(int64_t), st));
    const unsigned gA = (unsigned)((na + 255) / 256), gw = (unsigned)((na * 32 + 255) / 256);
    const SGeom *geom = (const SGeom *)c->cgeom.ptr;
    if (na > 0) {
        k_max_disp<<<gA, 256, 0, st>>>(na, c->pos.as<float>(), c->cand_ref.as<float>(),
                                       (unsigned long long *)disp_dev);
        k_filter<false><<<gw, 256, 0, st>>>(na, c->cand_off.as<int64_t>(), c->cand_key.as<uint64_t>(),
                                            c->pos.as<float>(), c->struct_of.as<int>(), geom, rcR * rcR, rcA * rcA,
                                            c->cand_flag.as<uint8_t>(), c->cand_rec.as<float4>(),
                                            c->cnt.as<int64_t>(), c->n_ang.as<int>(), nullptr, nullptr, nullptr,
                                            nullptr);
        CK(cudaGetLastError());
    }
    int rc = scan_exclusive(c, c->cnt.as<int64_t>(), na, c->nbr_off.as<int64_t>(), c->d_total.as<int64_t>());
    if (rc) return rc;
    if (na > 0) {
        k_filter<true><<<gw, 256, 0, st>>>(na, c->cand_off.as<int64_t>(), c->cand_key.as<uint64_t>(),
                                           c->pos.as<float>(), c->struct_of.as<int>(), geom, rcR * rcR, rcA * rcA,
                                           c->cand_flag.as<uint8_t>(), c->cand_rec.as<float4>(), nullptr,
                                           c->n_ang.as<int>(),
                                           c->nbr_off.as<int64_t>(), (float4 *)c->pair.ptr, c->shift.as<int32_t>(),
                                           c->cand_pidx.as<int>());
        if (Mc > 0)
            k_filter_rev<<<(unsigned)((Mc + 255) / 256), 256, 0, st>>>(Mc, c->cand_pidx.as<int>(),
                                                                      c->cand_rev.as<int>(), c->rev.as<int>());
        k_sum_int<<<(unsigned)std::min<int64_t>((na + 255) / 256, 1024), 256, 0, st>>>(na, c->n_ang.as<int>(), nang_dev);
        CK(cudaGetLastError());
    }
    int64_t tot[3] = {0, 0, 0};  // pairs, angular pairs, max squared displacement
    int herr = 0;
    CK(cudaMemcpyAsync(&tot[0], c->d_total.as<int64_t>(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tot[1], nang_dev, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) return c->fail(NEP_EINTERNAL, "candidate filter");
    double d2;
    std::memcpy(&d2, &tot[2], sizeof(double));
    // 2 d < s with a margin far above the rounding of the predicates (relative 1e-7 of r_c)
    if (!(2.0 * std::sqrt(d2) < (double)c->skin - 1e-5)) {
        moved_too_far = true;
        return NEP_OK;
    }
    c->n_pairs = tot[0];
    c->n_pairs_ang = tot[1];
    c->h_lists_ok = false;
    return host_lists ? fetch_host_lists(c) : NEP_OK;
}

// Host copies of the per-atom angular counts and CSR offsets (used by the host-side
// schedule builders); copied only when the lists changed since the last copy.
int fetch_host_lists(Ctx *c) {
    if (c->h_lists_ok) return NEP_OK;
    const int64_t na = c->n_atoms;
    c->h_nang.assign(na, 0);
    c->h_nbr_off.assign(na + 1, 0);
    if (na > 0) {
        CK(cudaMemcpy(c->h_nang.data(), c->n_ang.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(c->h_nbr_off.data(), c->nbr_off.ptr, sizeof(int64_t) * (na + 1), cudaMemcpyDeviceToHost));
    }
    c->h_lists_ok = true;
    return NEP_OK;
}

}  // namespace nep
