// Per-atom kernels of the NEP loss + parameter-gradient pass (descriptors, network, pair
// gradients, and the adjoint).  Persistent over a static species-sorted schedule: each
// warp owns a contiguous range of work positions and processes them in batches of G = 32/SW
// atoms of one species, one group of SW lanes per atom, so that the ~15-20 angular
// and ~60-80 radial neighbours of an atom keep most lanes busy.
//
// Forward (k_fwd_desc -> k_net_fwd -> k_fwd_pair):
//   A_nlm = sum_j g^A_n(r_ij) Y_lm(r^_ij)          pair geometry staged in shared memory,
//                                                   lanes own (l, m) outputs
//   q_n   = sum_j sum_k c^{t_i t_j}_{nk} f_k(r_ij)  (one species: through the sums
//                                                   S_k = sum_j f_k(r_ij), q being linear in c)
//   q_nl  = sum_m A_nlm^2, q4_n, q5_n               (Methods, Eq. "q3b"; 4-/5-body readings)
//   E_i   = w1 . tanh(W0 q~ - b0) - b1              (Eq. "ann"), e = dE_i/dq~
//   G_p   = dE_i/dd_p                               pair gradients, written per pair
// Adjoint (k_adj_jvp -> k_net_rev -> k_adj_cg), for cotangents fbar = dL/dF,
// ebar = dL/dE_s, wbar = dL/dW_s:
//   lambda_p = fbar_i - fbar_j - wbar_s d_p
//   dq_i = sum_p (dq_i/dd_p) lambda_p               forward-mode JVP of the descriptors
//   reverse through the network (tanh', tanh'') -> per-atom vectors for the network
//   gradient, abar = dJ/dq (tiled products over chunks of atoms of one species);
//   then dJ/dc (radial part factorised over species sums, angular part per pair).
//
// Work layout.  Per-pair quantities are computed one pair per lane; reductions over
// the pairs of an atom go through rows staged in shared memory and read by lanes that
// own outputs, in a fixed order:
//   * angular moments and their JVP: lanes own (l, m);
//   * radial species sums S^b_k of the adjoint (more than one species): lanes own k and
//     walk their atom's rows, which come sorted by neighbour species, adding each species
//     run into the atom's S^b (one species: every lane sums its own pairs, one reduction
//     per atom); the forward's radial descriptor takes each pair's g_n directly;
//   * angular coefficient gradient: all 32 lanes own (n, k-range) tiles of the current
//     (t_i, t_j) block and walk the rows of every atom of the batch; a species change
//     flushes the tile into the warp's shared accumulator (one species and a small block:
//     every lane sums the whole block over its own pairs in registers instead, and the
//     lanes reduce it once per warp).
// Per-atom matrices that every pair of an atom reads (dE/dA, dJ/dA) are stored [lm][n]
// with n padded to a multiple of 4, and the coefficient rows c[n][k] are 16-byte-aligned
// copies in the parameter buffer, so both are read with 128-bit loads.
// FP32 arithmetic with FP32 accumulation inside an atom; no floating-point atomics, so
// results are bit-reproducible for a fixed launch shape.
#pragma once

#include "nep_ctx.cuh"

namespace nep {

// ============================================================================= helpers

// v[i] for a compile-time array of length K; the index is clamped so that unrolled,
// compile-time-dead terms never name an element past the end.
template <int K>
__device__ __forceinline__ float at_k(const float *v, int i) { return v[i < K ? i : K - 1]; }

// g_n = sum_k c[n][k] f_k, n < N, from 16-byte-aligned rows of round4(K) floats.
template <int N, int K>
__device__ __forceinline__ void contract_c(const float *c, const float *f, float *g) {
    constexpr int K4 = round4(K);
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const float4 *r = reinterpret_cast<const float4 *>(c + n * K4);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < K4 / 4; ++q) {
            const float4 v = __ldg(r + q);
            if (4 * q + 0 < K) s += v.x * at_k<K>(f, 4 * q + 0);
            if (4 * q + 1 < K) s += v.y * at_k<K>(f, 4 * q + 1);
            if (4 * q + 2 < K) s += v.z * at_k<K>(f, 4 * q + 2);
            if (4 * q + 3 < K) s += v.w * at_k<K>(f, 4 * q + 3);
        }
        g[n] = s;
    }
}

// g_n = sum_k c[n][k] f_k and gp_n = sum_k c[n][k] fp_k from the same rows.
template <int N, int K>
__device__ __forceinline__ void contract_c2(const float *c, const float *f, const float *fp, float *g, float *gp) {
    constexpr int K4 = round4(K);
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const float4 *r = reinterpret_cast<const float4 *>(c + n * K4);
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int q = 0; q < K4 / 4; ++q) {
            const float4 v = __ldg(r + q);
            const float cv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * q + e < K) {
                    s0 += cv[e] * at_k<K>(f, 4 * q + e);
                    s1 += cv[e] * at_k<K>(fp, 4 * q + e);
                }
            }
        }
        g[n] = s0;
        gp[n] = s1;
    }
}

// Stores v[0..N) as a row of round4(N) floats (zero padding) with 128-bit stores.
template <int N>
__device__ __forceinline__ void store_row4(float *dst, const float *v) {
    constexpr int N4 = round4(N);
    float4 *d = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int q = 0; q < N4 / 4; ++q)
        d[q] = make_float4(4 * q + 0 < N ? at_k<N>(v, 4 * q + 0) : 0.0f, 4 * q + 1 < N ? at_k<N>(v, 4 * q + 1) : 0.0f,
                           4 * q + 2 < N ? at_k<N>(v, 4 * q + 2) : 0.0f, 4 * q + 3 < N ? at_k<N>(v, 4 * q + 3) : 0.0f);
}

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
// (< wend): group g reads the work record of position base + g, so the loads of all groups
// are one round trip together.  Returns the species ti, the batch size nb and this group's
// atom with its pair range and structure (the batch's first atom, with no pairs, for
// groups beyond nb).
struct BatchAtom {
    int ti, nb, i, beg, nRad, nAng, s;
};
template <int SW>
__device__ __forceinline__ BatchAtom load_batch(const AtomArgs &a, int base, int wend, int lane) {
    constexpr int G = 32 / SW;
    const int grp = lane / SW;
    const int q = base + grp;
    const bool valid = grp < G && q < wend;
    const int4 r = valid ? __ldg(a.rec + q) : make_int4(-1, 0, 0, 0);
    const int2 r2 = valid ? __ldg(a.rec2 + q) : make_int2(-1, 0);
    BatchAtom b;
    b.ti = __shfl_sync(FULL, r2.x, 0);
    const unsigned same = __ballot_sync(FULL, r2.x == b.ti);
    unsigned gm = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) gm |= ((same >> (g * SW)) & 1u) << g;
    b.nb = min(G, __ffs(~gm) - 1);
    const int i0 = __shfl_sync(FULL, r.x, 0), beg0 = __shfl_sync(FULL, r.y, 0), s0 = __shfl_sync(FULL, r2.y, 0);
    const bool act = grp < b.nb;
    b.i = act ? r.x : i0;
    b.beg = act ? r.y : beg0;
    b.nRad = act ? r.z : 0;
    b.nAng = act ? r.w : 0;
    b.s = act ? r2.y : s0;
    return b;
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

// Species sums over an atom's radial neighbours, several species: the group's lanes each
// computed the C values of one pair and staged them in rows[SW][C + 1] (the species bits in
// the last slot); lane sl owns columns sl, sl + SW, ... and walks the cnt rows in order,
// adding each species run into S[b][0..C).  v / bcur carry the open run across chunks.
template <int C, int SW>
__device__ __forceinline__ void walk_species_rows(const float (*rows)[C + 1], int cnt, int sl, float *S, float *v,
                                                  int &bcur) {
    constexpr int RC = (C + SW - 1) / SW;
#pragma unroll 2
    for (int pp = 0; pp < cnt; ++pp) {
        const float *row = rows[pp];
        const int t = __float_as_int(row[C]);
        if (t != bcur) {
            if (bcur >= 0) {
#pragma unroll
                for (int j = 0; j < RC; ++j)
                    if (sl + j * SW < C) S[bcur * C + sl + j * SW] += v[j];
            }
#pragma unroll
            for (int j = 0; j < RC; ++j) v[j] = 0.0f;
            bcur = t;
        }
#pragma unroll
        for (int j = 0; j < RC; ++j)
            if (sl + j * SW < C) v[j] += row[sl + j * SW];
    }
}

template <int C, int SW>
__device__ __forceinline__ void close_species_run(int sl, float *S, const float *v, int bcur) {
    constexpr int RC = (C + SW - 1) / SW;
    if (bcur >= 0) {
#pragma unroll
        for (int j = 0; j < RC; ++j)
            if (sl + j * SW < C) S[bcur * C + sl + j * SW] += v[j];
    }
}

// The l = 2 moments (m = -2..2) of channel n from a [lm][n] matrix with row stride NAP.
template <int NAP>
__device__ __forceinline__ void l2_block(const float *M, int n, float *a) {
#pragma unroll
    for (int m = 0; m < 5; ++m) a[m] = M[(3 + m) * NAP + n];
}

// ============================================================================= layouts

// Forward, stage 1 (k_fwd_desc): descriptors.
template <class S, int SW>
struct DescL {
    static constexpr int G = 32 / SW;
    static constexpr int NAP = round4(S::NA);
    static constexpr int NLMO = (L3 + SW - 1) / SW;  // (l, m) outputs owned per lane
    struct __align__(16) Atom {
        float A[L3 * NAP];  // A_nlm at [lm][n]
        float q[S::ND];
    };
    struct __align__(16) Mom {
        float g[G][SW][NAP];  // g^A_n of each lane's pair
        float Y[G][SW][L3];
    };
    Atom at[G];
    Mom st;
    // runtime tail (floats): S[G][KR] (one species)
    __host__ __device__ static size_t tail(int T, int NN) { return (size_t)G * S::KR; }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(DescL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

// Forward, stage 3 (k_fwd_pair): pair gradients.
template <class S, int SW>
struct PairL {
    static constexpr int G = 32 / SW;
    static constexpr int NAP = round4(S::NA);
    static constexpr int NLMO = (L3 + SW - 1) / SW;
    struct __align__(16) Atom {
        float A[L3 * NAP];   // A_nlm at [lm][n]
        float Ah[L3 * NAP];  // dE_i/dA_nlm at [lm][n]
        float b[S::ND];
        float G4[S::NA * 5];
    };
    Atom at[G];
    // runtime tail (floats): beta[G][T][KR]
    __host__ __device__ static size_t tail(int T, int NN) { return (size_t)G * T * S::KR; }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(PairL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

// Adjoint, stage 1 (k_adj_jvp): the JVP of the descriptors.
template <class S, int SW>
struct JvpL {
    static constexpr int G = 32 / SW;
    static constexpr int NAP = round4(S::NA);
    static constexpr int NLMO = (L3 + SW - 1) / SW;
    struct __align__(16) Atom {
        float A[L3 * NAP];  // A_nlm at [lm][n]
        float D[L3 * NAP];  // dA_nlm, the JVP of the moments, at [lm][n]
        float dqt[S::ND];
        float G4[S::NA * 5];
    };
    struct __align__(16) Jvp {
        float g[G][SW][NAP];   // g^A_n
        float gp[G][SW][NAP];  // (r^.lambda) dg^A_n/dr
        float Y[G][SW][L3];
        float P[G][SW][L3];    // grad Y_lm . p, p the part of lambda / r normal to r^
    };
    struct __align__(16) Rad {
        float f[G][SW][2 * S::KR + 1];  // f_k, (r^.lambda) f'_k, then the species bits
    };
    Atom at[G];
    union {
        Jvp j;
        Rad r;
    } st;
    // runtime tail: Sr[G][T][2 KR]
    __host__ __device__ static size_t tail(int T, int NN) { return 2 * (size_t)G * T * S::KR; }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(JvpL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

// Adjoint, stage 3 (k_adj_cg): dJ/dA and the coefficient gradient.
template <class S, int SW>
struct CgL {
    static constexpr int G = 32 / SW;
    static constexpr int NAP = round4(S::NA);
    static constexpr int NLMO = (L3 + SW - 1) / SW;
    struct __align__(16) Atom {
        float A[L3 * NAP];   // A_nlm at [lm][n]
        float D[L3 * NAP];   // dA, then dJ/dA in place
        float Ah[L3 * NAP];  // dE_i/dA
        float b[S::ND];
        float ab[S::ND];
        float G4[S::NA * 5];
        float H4[S::NA * 5];
        float ad[S::NA];  // sum_m A_n1m dA_n1m (read by every l = 1 lane before dA is overwritten)
    };
    struct __align__(16) Cg {
        float2 ab[G][SW][S::NA];  // (alpha_n, beta_n) of each lane's pair
        float2 ff[G][SW][S::KA];  // (f_k, f'_k)
        int t[G][SW];             // species of the neighbour
    };
    Atom at[G];
    Cg st;
    // runtime tail: Sr[G][T][2 KR], accR[T][NCR], accA[T][NCA]
    __host__ __device__ static size_t tail(int T, int NN) {
        return 2 * (size_t)G * T * S::KR + (size_t)T * (S::NCR + S::NCA);
    }
    __host__ __device__ static size_t bytes(int T, int NN) {
        return ((sizeof(CgL) + sizeof(float) * tail(T, NN)) + 15) & ~(size_t)15;
    }
};

// ============================================================================= adjoint
// Three stages, for cotangents fbar = dL/dF, ebar = dL/dE_s, wbar = dL/dW_s:
//   k_adj_jvp  (per atom)  lambda_p = fbar_i - fbar_j - wbar_s d_p; the JVP dq~ of the
//                          descriptors along lambda; stores dq~, dA and the radial
//                          species sums S^b_k, S'^b_k;
//   k_net_rev  (per chunk of atoms of one species, tiled products) the reverse pass through
//                          the network: zeta, u, omega and abar = dJ/dq~, b = dE/dq~;
//   k_adj_cg   (per atom)  dJ/dA and the gradient into the coefficients c.

// Copy of N floats of per-atom state (written by an earlier stage) by the SW lanes of a
// group: up to eight loads of a lane are issued before their stores, so the copy costs
// about N / (8 SW) memory round trips instead of N / SW.  st(e, value) places element e.
template <int N, int SW, class St>
__device__ __forceinline__ void gather_rows(const float *src, int sl, St st) {
    constexpr int IT = (N + SW - 1) / SW;
    constexpr int B = IT < 8 ? IT : 8;
#pragma unroll
    for (int i0 = 0; i0 < IT; i0 += B) {
        float v[B];
#pragma unroll
        for (int it = 0; it < B; ++it) {
            const int e = sl + (i0 + it) * SW;
            v[it] = (i0 + it < IT && e < N) ? __ldg(src + e) : 0.0f;
        }
#pragma unroll
        for (int it = 0; it < B; ++it) {
            const int e = sl + (i0 + it) * SW;
            if (i0 + it < IT && e < N) st(e, v[it]);
        }
    }
}

// The same for a run-time length n, eight loads per lane in flight at a time.
template <int SW, class St>
__device__ __forceinline__ void gather_rows_n(const float *src, int n, int sl, St st) {
    for (int e0 = 0; e0 < n; e0 += 8 * SW) {
        float v[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int e = e0 + sl + it * SW;
            v[it] = e < n ? __ldg(src + e) : 0.0f;
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int e = e0 + sl + it * SW;
            if (e < n) st(e, v[it]);
        }
    }
}

// Block-wide staging of n elements by NT threads, eight loads per thread in flight:
// ld(e) returns element e (or the padding value), st(e, value) places it.
template <int NT, class Ld, class St>
__device__ __forceinline__ void block_stage(int n, Ld ld, St st) {
    for (int e0 = 0; e0 < n; e0 += 8 * NT) {
        float v[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int e = e0 + (int)threadIdx.x + it * NT;
            v[it] = e < n ? ld(e) : 0.0f;
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int e = e0 + (int)threadIdx.x + it * NT;
            if (e < n) st(e, v[it]);
        }
    }
}

// Loads a [lm][n]-packed per-atom matrix (NA x 24 floats) into a [lm][NAP] shared row set.
template <int NA, int NAP, int SW>
__device__ __forceinline__ void load_lm_rows(const float *src, float *dst, int sl) {
    gather_rows<L3 * NA, SW>(src, sl, [&](int e, float x) {
        const int lm = e / NA, n = e - lm * NA;
        dst[lm * NAP + n] = x;
    });
}

// lambda_p of a pair (record pd, neighbour j) of an atom with cotangent fbi and structure wbar
__device__ __forceinline__ void pair_lambda(const AtomArgs &a, float4 pd, float fbx, float fby, float fbz,
                                            const float *Wb, float &lx, float &ly, float &lz) {
    const float4 fbj = a.fbar[pair_j(pd)];
    lx = fbx - fbj.x - (Wb[0] * pd.x + Wb[1] * pd.y + Wb[2] * pd.z);
    ly = fby - fbj.y - (Wb[3] * pd.x + Wb[4] * pd.y + Wb[5] * pd.z);
    lz = fbz - fbj.z - (Wb[6] * pd.x + Wb[7] * pd.y + Wb[8] * pd.z);
}

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(128, VAR == 0 ? 4 : 5) k_adj_jvp(AtomArgs a) {
    grid_dep_wait();
    grid_dep_launch();
    using L = JvpL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int G = L::G, NAP = L::NAP, NLMO = L::NLMO;
    constexpr int KR4 = round4(KR), KA4 = round4(KA);
    constexpr int VR2 = pow2ceil(2 * KR);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *tail = base_ptr + sizeof(L) / sizeof(float);
    float *Sr = tail + grp * T * 2 * KR;  // [T][2 KR] S^b_k | S'^b_k of this group

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);
    const float *scale = a.par + po.scale;

    for (int bp = wbeg; bp < wend;) {
        const BatchAtom ba = load_batch<SW>(a, bp, wend, lane);
        const int ti = ba.ti, nb = ba.nb, i = ba.i;
        const bool act = grp < nb;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
        const float *cRi = a.par + po.cRp + (size_t)ti * T * NR * KR4;
        const float *cAi = a.par + po.cAp + (size_t)ti * T * NA * KA4;
        const int s = ba.s;
        const int64_t beg = ba.beg;
        const int nRad = ba.nRad;
        const int nAng = ba.nAng;
        const int maxR = __reduce_max_sync(FULL, nRad);
        const int maxA = __reduce_max_sync(FULL, nAng);
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their pair records into L2
            const int4 nr = __ldg(a.rec + bp + grp);
            prefetch_l2(a.pair + nr.y, sizeof(float4) * (size_t)nr.z, sl, SW);
        }
        load_lm_rows<NA, NAP, SW>(a.st_A + (size_t)wi * NA * L3, at.A, sl);
        const float4 *prs = a.pair + beg;
        const float4 fbi = a.fbar[i];
        const float fbx = fbi.x, fby = fbi.y, fbz = fbi.z;
        float Wb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Wb[k] = a.wbar[(size_t)s * 9 + k];
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
                    const int tj = pair_t(pd);
                    float lx, ly, lz;
                    pair_lambda(a, pd, fbx, fby, fbz, Wb, lx, ly, lz);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    const float r = r2 * rinv;
                    const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
                    const float rl = ux * lx + uy * ly + uz * lz;
                    const float px = (lx - rl * ux) * rinv, py = (ly - rl * uy) * rinv, pz = (lz - rl * uz) * rinv;
                    float f[KA], fp[KA], g[NA], gp[NA];
                    basis_val_der<KA>(r, a.inv_rcA, f, fp);
                    contract_c2<NA, KA>(cAi + tj * NA * KA4, f, fp, g, gp);
#pragma unroll
                    for (int n = 0; n < NA; ++n) gp[n] *= rl;
                    store_row4<NA>(sm.st.j.g[grp][sl], g);
                    store_row4<NA>(sm.st.j.gp[grp][sl], gp);
                    float *Yr = sm.st.j.Y[grp][sl], *Pr = sm.st.j.P[grp][sl];
                    ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                        Yr[lm] = Y;
                        Pr[lm] = gx * px + gy * py + gz * pz;
                    });
                }
                __syncwarp();
                const int cnt = min(SW, nAng - c0);
#pragma unroll 2
                for (int pp = 0; pp < cnt; ++pp) {
                    float gv[NAP], gpv[NAP];
                    load_row<NAP>(sm.st.j.g[grp][pp], gv);
                    load_row<NAP>(sm.st.j.gp[grp][pp], gpv);
#pragma unroll
                    for (int jj = 0; jj < NLMO; ++jj) {
                        const int lm = sl + jj * SW;
                        if (lm < L3) {
                            const float y = sm.st.j.Y[grp][pp][lm], ps = sm.st.j.P[grp][pp][lm];
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
                    store_row4<NA>(at.D + lm * NAP, accd[jj]);
                    if (act) {
#pragma unroll
                        for (int n = 0; n < NA; ++n) a.st_D[(size_t)wi * NA * L3 + lm * NA + n] = accd[jj][n];
                    }
                }
            }
        }

        // ---------------------------------------------------------------- radial JVP species sums
        for (int e = sl; e < T * 2 * KR; e += SW) Sr[e] = 0.0f;
        __syncwarp();
        if (T == 1) {  // one species: every lane sums its own pairs, one reduction per atom
            float v[VR2];
#pragma unroll
            for (int k = 0; k < VR2; ++k) v[k] = 0.0f;
            float4 nxt = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nRad);
                if (k < nRad) {
                    float lx, ly, lz;
                    pair_lambda(a, pd, fbx, fby, fbz, Wb, lx, ly, lz);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    const float rl = (pd.x * lx + pd.y * ly + pd.z * lz) * rinv;
                    float f[KR], fp[KR];
                    basis_val_der<KR>(r2 * rinv, a.inv_rcR, f, fp);
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) {
                        v[kk] += f[kk];
                        v[KR + kk] += rl * fp[kk];
                    }
                }
            }
            if (__any_sync(FULL, nRad > 0)) flush_groups<VR2, SW>(v, Sr, 2 * KR, nRad > 0, lane, false);
        } else {
            constexpr int RC2 = (2 * KR + SW - 1) / SW;
            float v[RC2];
            int bcur = -1;
            float4 nxt = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nRad);
                if (k < nRad) {
                    float lx, ly, lz;
                    pair_lambda(a, pd, fbx, fby, fbz, Wb, lx, ly, lz);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    const float rl = (pd.x * lx + pd.y * ly + pd.z * lz) * rinv;
                    float *row = sm.st.r.f[grp][sl];
                    float fp[KR];
                    basis_val_der<KR>(r2 * rinv, a.inv_rcR, row, fp);
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) row[KR + kk] = rl * fp[kk];
                    row[2 * KR] = __int_as_float(pair_t(pd));
                }
                __syncwarp();
                walk_species_rows<2 * KR, SW>(sm.st.r.f[grp], min(SW, nRad - c0), sl, Sr, v, bcur);
                __syncwarp();
            }
            close_species_run<2 * KR, SW>(sl, Sr, v, bcur);
        }
        __syncwarp();
        if (act)
            for (int e = sl; e < T * 2 * KR; e += SW) a.st_S[(size_t)wi * T * 2 * KR + e] = Sr[e];

        // ---------------------------------------------------------------- JVP of the descriptors
        for (int n = sl; n < NA; n += SW) {
            float a2[5], Mt[6], M2[6], pr[5];
            l2_block<NAP>(at.A, n, a2);
            l2_matrix(a2, Mt);
            sym_prod(Mt, Mt, M2);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.G4[n * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
        }
        for (int n = sl; n < NR; n += SW) {
            float d = 0.0f;
            for (int bb = 0; bb < T; ++bb) {
                const float *cr = cRi + (bb * NR + n) * KR4;
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) d += __ldg(cr + kk) * Sr[bb * 2 * KR + KR + kk];
            }
            at.dqt[n] = d * scale[n];
        }
        for (int e = sl; e < 4 * NA; e += SW) {
            const int n = e % NA, l = e / NA + 1;
            float s2 = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) {
                const int lm = l * l - 1 + m;
                s2 += at.A[lm * NAP + n] * at.D[lm * NAP + n];
            }
            const int v = NR + (l - 1) * NA + n;
            at.dqt[v] = 2.0f * s2 * scale[v];
        }
        __syncwarp();
        for (int n = sl; n < NA; n += SW) {
            float d2[5];
            l2_block<NAP>(at.D, n, d2);
            float d4 = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) d4 += at.G4[n * 5 + m] * d2[m];
            at.dqt[NR + 4 * NA + n] = d4 * scale[NR + 4 * NA + n];
            const float x0 = at.A[n], x1 = at.A[NAP + n], x2 = at.A[2 * NAP + n];
            const float q1 = x0 * x0 + x1 * x1 + x2 * x2;
            const float ad = x0 * at.D[n] + x1 * at.D[NAP + n] + x2 * at.D[2 * NAP + n];
            at.dqt[NR + 5 * NA + n] = 4.0f * q1 * ad * scale[NR + 5 * NA + n];
        }
        __syncwarp();
        if (act)
            for (int v = sl; v < ND; v += SW) a.dqt[(size_t)wi * ND + v] = at.dqt[v];
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------- network reverse
// Per chunk of <= 128 work positions of one species t, in tiles of 64 atoms (16 for chunks of
// at most 16) (Eq. "ann"):
//   v = W0 dq~,  h' = 1 - h^2,  h'' = -2 h h',
//   zeta = ebar w1 h' + w1 h'' v,  u = w1 h',  omega = ebar h + h' v,
//   abar = s (W0^T zeta)   (b = s (W0^T u) comes from the network forward pass).
// 256 threads as 16 x 16; each owns 4 atoms x 4 columns of a 64 x 64 output block, and the
// operands come from shared memory with 128-bit loads (atoms along the fast axis).
constexpr int NETR = 64;  // atoms per tile of chunks longer than 16 work positions

// RX consecutive floats of a transposed tile row (RX = 4: one 128-bit load).
template <int RX>
__device__ __forceinline__ void ld_rows(const float *p, float *v) {
    if constexpr (RX == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
#pragma unroll
        for (int x = 0; x < RX; ++x) v[x] = p[x];
    }
}

template <class S, int RX>
__host__ __device__ inline size_t net_rev_smem(int NN) {
    constexpr int R = 16 * RX;
    const size_t NDQ = round4(S::ND), NNP = round4(NN);
    return sizeof(float) * (NDQ * R + NNP * R + (size_t)S::ND * NNP + (size_t)NN * NDQ);
}

template <class S, int RX>
__global__ void __launch_bounds__(256) k_net_rev(AtomArgs a) {
    constexpr int R = 16 * RX;  // tile rows: 16 row groups of RX
    grid_dep_wait();
    grid_dep_launch();
    constexpr int ND = S::ND, NDQ = round4(ND);
    extern __shared__ __align__(16) float smn[];
    const int NN = a.NN, NNP = round4(NN), T = a.T;
    float *Q = smn;                 // [NDQ][R] dq~, transposed
    float *Z = Q + NDQ * R;      // [NNP][R] zeta, transposed
    float *Wt = Z + NNP * R;     // [ND][NNP]  W0^T of the species
    float *Wn = Wt + ND * NNP;      // [NN][NDQ]  W0 of the species
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int rc0 = a.chunks[blockIdx.x], rc1 = a.chunks[blockIdx.x + 1];
    if (rc0 >= rc1) return;
    const int t = __ldg(a.rec2 + rc0).x;
    const ParOff po = par_offsets(T, NN, S::NR, S::KR, S::NA, S::KA);
    const float *W0 = a.par + po.w0 + (size_t)t * NN * ND;
    const float *W0T = a.par + po.w0t + (size_t)t * ND * NN;
    const float *w1 = a.par + po.w1 + (size_t)t * NN;
    const float *scale = a.par + po.scale;
    block_stage<256>(
        ND * NNP,
        [&](int e) {
            const int k = e / NNP, mu = e - k * NNP;
            return mu < NN ? __ldg(W0T + (size_t)k * NN + mu) : 0.0f;
        },
        [&](int e, float x) { Wt[e] = x; });
    block_stage<256>(
        NN * NDQ,
        [&](int e) {
            const int mu = e / NDQ, v = e - mu * NDQ;
            return v < ND ? __ldg(W0 + (size_t)mu * ND + v) : 0.0f;
        },
        [&](int e, float x) { Wn[e] = x; });
    for (int rb = rc0; rb < rc1; rb += R) {
        const int nr = min(R, rc1 - rb);
        __syncthreads();  // the weights are staged; the previous tile is done with Q, Z, U
        block_stage<256>(
            R * NDQ,
            [&](int e) {
                const int r = e / NDQ, k = e - r * NDQ;
                return (r < nr && k < ND) ? __ldg(a.dqt + (size_t)(rb + r) * ND + k) : 0.0f;
            },
            [&](int e, float x) {
                const int r = e / NDQ, k = e - r * NDQ;
                Q[k * R + r] = x;
            });
        __syncthreads();
        const int r0 = ty * RX;
        for (int cb = 0; cb < NNP; cb += 64) {
            const int mu0 = cb + tx * 4;
            if (mu0 < NNP) {
                float acc[RX][4];
#pragma unroll
                for (int x = 0; x < RX; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
#pragma unroll 7
                for (int k = 0; k < ND; ++k) {
                    float q[RX];
                    ld_rows<RX>(Q + k * R + r0, q);
                    const float4 w4 = *reinterpret_cast<const float4 *>(Wt + k * NNP + mu0);
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < RX; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] += q[x] * wv[y];
                }
#pragma unroll
                for (int x = 0; x < RX; ++x) {
                    const int r = r0 + x;
                    const bool row = r < nr;
                    const int wpos = rb + (row ? r : 0);
                    const float eb = row ? a.ebar[__ldg(a.rec2 + wpos).y] : 0.0f;
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int mu = mu0 + y;
                        float ze = 0.0f;
                        if (row && mu < NN) {
                            const float h = a.st_h[(size_t)wpos * NN + mu];
                            const float wo = w1[mu];
                            const float hp = 1.0f - h * h;
                            const float hpp = -2.0f * h * hp;
                            ze = eb * wo * hp + wo * hpp * acc[x][y];
                            a.zt[(size_t)wpos * NN + mu] = ze;
                            a.ut[(size_t)wpos * NN + mu] = wo * hp;
                            a.om[(size_t)wpos * NN + mu] = eb * h + hp * acc[x][y];
                        }
                        Z[mu * R + r] = ze;
                    }
                }
            }
        }
        __syncthreads();
        for (int cb = 0; cb < NDQ; cb += 64) {
            const int v0 = cb + tx * 4;
            if (v0 < NDQ) {
                float aa[RX][4];
#pragma unroll
                for (int x = 0; x < RX; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) aa[x][y] = 0.0f;
#pragma unroll 5
                for (int mu = 0; mu < NN; ++mu) {
                    float z[RX];
                    ld_rows<RX>(Z + mu * R + r0, z);
                    const float4 w4 = *reinterpret_cast<const float4 *>(Wn + mu * NDQ + v0);
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < RX; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) aa[x][y] += z[x] * wv[y];
                }
#pragma unroll
                for (int x = 0; x < RX; ++x) {
                    const int r = r0 + x;
                    if (r < nr) {
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const int v = v0 + y;
                            if (v < ND) a.st_ab[(size_t)(rb + r) * ND + v] = aa[x][y] * scale[v];
                        }
                    }
                }
            }
        }
    }
}

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(128, VAR == 0 ? 4 : 5) k_adj_cg(AtomArgs a) {
    grid_dep_wait();
    grid_dep_launch();
    using L = CgL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int NCR = S::NCR, NCA = S::NCA, NC = S::NC;
    constexpr int G = L::G, NAP = L::NAP, NLMO = L::NLMO;
    // angular coefficient-gradient tiles: lane -> (n, k-range of width TW), 32 lanes
    constexpr int NKT = 32 / NA;
    constexpr int TW = (KA + NKT - 1) / NKT;
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *tail = base_ptr + sizeof(L) / sizeof(float);
    float *Sr = tail + grp * T * 2 * KR;       // [T][2 KR] S^b_k | S'^b_k of this group
    float *accR = tail + G * T * 2 * KR;       // [T][NCR] (warp)
    float *accA = accR + T * NCR;              // [T][NCA] (warp)
    const int tn = lane % NA, tk0 = (lane / NA) * TW;
    const bool tile_own = lane / NA < NKT && tk0 < KA;

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];

    int cur_t = -1;
    // One species (and a coefficient block of at most 64 values): every lane keeps the whole
    // (0, 0) block of the angular coefficient gradient for its own pairs, across all the
    // warp's atoms, and the group lanes reduce it once at the end of the warp's range.
    constexpr bool REG1 = S::NCA <= 64;
    constexpr int V1 = REG1 ? pow2ceil(NCA) : 1;
    const bool one_species = REG1 && T == 1;
    float X1[V1];
#pragma unroll
    for (int e = 0; e < V1; ++e) X1[e] = 0.0f;
    // open (t_i, t_j) tile of the angular coefficient gradient, carried across batches
    float X[TW];
#pragma unroll
    for (int jj = 0; jj < TW; ++jj) X[jj] = 0.0f;
    int xb = -1;
    auto close_tile = [&]() {
        if (xb >= 0 && tile_own) {
#pragma unroll
            for (int jj = 0; jj < TW; ++jj)
                if (tk0 + jj < KA) accA[xb * NCA + tn * KA + tk0 + jj] += X[jj];
        }
#pragma unroll
        for (int jj = 0; jj < TW; ++jj) X[jj] = 0.0f;
    };
    auto flush_slot = [&](int t) {
        float *dst = a.cpart + (size_t)(w + t) * T * NC;
        for (int bb = 0; bb < T; ++bb) {
            for (int e = lane; e < NCR; e += 32) dst[(size_t)bb * NC + e] = accR[bb * NCR + e];
            for (int e = lane; e < NCA; e += 32) dst[(size_t)bb * NC + NCR + e] = accA[bb * NCA + e];
        }
    };

    for (int bp = wbeg; bp < wend;) {
        const BatchAtom ba = load_batch<SW>(a, bp, wend, lane);
        const int ti = ba.ti, nb = ba.nb, i = ba.i;
        const bool act = grp < nb;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
        if (ti != cur_t) {
            __syncwarp();
            close_tile();
            xb = -1;
            __syncwarp();
            if (cur_t >= 0) flush_slot(cur_t);
            for (int e = lane; e < T * NCR; e += 32) accR[e] = 0.0f;
            for (int e = lane; e < T * NCA; e += 32) accA[e] = 0.0f;
            cur_t = ti;
            __syncwarp();
        }
        const int s = ba.s;
        const int64_t beg = ba.beg;
        const int nAng = ba.nAng;
        const int maxA = __reduce_max_sync(FULL, nAng);
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their angular records into L2
            const int4 nr = __ldg(a.rec + bp + grp);
            prefetch_l2(a.pair + nr.y, sizeof(float4) * (size_t)nr.w, sl, SW);
        }

        // ---------------------------------------------------------------- state of the earlier stages
        load_lm_rows<NA, NAP, SW>(a.st_A + (size_t)wi * NA * L3, at.A, sl);
        load_lm_rows<NA, NAP, SW>(a.st_D + (size_t)wi * NA * L3, at.D, sl);
        gather_rows<ND, SW>(a.st_b + (size_t)wi * ND, sl, [&](int v, float x) { at.b[v] = x; });
        gather_rows<ND, SW>(a.st_ab + (size_t)wi * ND, sl, [&](int v, float x) { at.ab[v] = x; });
        gather_rows_n<SW>(a.st_S + (size_t)wi * T * 2 * KR, T * 2 * KR, sl,
                          [&](int e, float x) { Sr[e] = act ? x : 0.0f; });
        __syncwarp();
        for (int n = sl; n < NA; n += SW) {
            float a2[5], d2[5], Mt[6], dMt[6], M2[6], Pm[6], pr[5];
            l2_block<NAP>(at.A, n, a2);
            l2_block<NAP>(at.D, n, d2);
            l2_matrix(a2, Mt);
            l2_matrix(d2, dMt);
            sym_prod(Mt, Mt, M2);
            l2_project(M2, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.G4[n * 5 + m] = 3.0f * KAPPA_REAL * pr[m];
            sym_prod(Mt, dMt, Pm);
            l2_project(Pm, pr);
#pragma unroll
            for (int m = 0; m < 5; ++m) at.H4[n * 5 + m] = 6.0f * KAPPA_REAL * pr[m];
            at.ad[n] = at.A[n] * at.D[n] + at.A[NAP + n] * at.D[NAP + n] + at.A[2 * NAP + n] * at.D[2 * NAP + n];
        }
        __syncwarp();

        // ---------------------------------------------------------------- dE/dA and dJ/dA (in place of dA)
#pragma unroll
        for (int jj = 0; jj < NLMO; ++jj) {
            const int lm = sl + jj * SW;
            if (lm < L3) {
                const int l = l_of_lm(lm);
                float ah[NA], xr[NA];
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float av = at.A[lm * NAP + n], dv = at.D[lm * NAP + n];
                    const float x0 = at.A[n], x1 = at.A[NAP + n], x2 = at.A[2 * NAP + n];
                    const float q1 = x0 * x0 + x1 * x1 + x2 * x2;
                    const int v3 = NR + (l - 1) * NA + n;
                    float h = 2.0f * at.b[v3] * av;
                    float x = 2.0f * at.ab[v3] * av + 2.0f * at.b[v3] * dv;
                    if (l == 2) {
                        h += at.b[NR + 4 * NA + n] * at.G4[n * 5 + lm - 3];
                        x += at.ab[NR + 4 * NA + n] * at.G4[n * 5 + lm - 3] + at.b[NR + 4 * NA + n] * at.H4[n * 5 + lm - 3];
                    }
                    if (l == 1) {
                        const int v5 = NR + 5 * NA + n;
                        h += at.b[v5] * 4.0f * q1 * av;
                        x += at.ab[v5] * 4.0f * q1 * av + at.b[v5] * (8.0f * at.ad[n] * av + 4.0f * q1 * dv);
                    }
                    ah[n] = h;
                    xr[n] = x;
                }
                store_row4<NA>(at.Ah + lm * NAP, ah);
                store_row4<NA>(at.D + lm * NAP, xr);  // only this lane reads or writes row lm here
            }
        }
        const float4 *prs = a.pair + beg;
        const float4 fbi = a.fbar[i];
        const float fbx = fbi.x, fby = fbi.y, fbz = fbi.z;
        float Wb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Wb[k] = a.wbar[(size_t)s * 9 + k];
        __syncwarp();

        // ---------------------------------------------------------------- radial coefficient gradient
        // accR[b][n][k] += abar_n S^b_k + b_n S'^b_k for each atom of the batch in turn, all 32
        // lanes on one atom: lane -> (b, n), the K_R products of the row unrolled
#pragma unroll 1
        for (int g2 = 0; g2 < nb; ++g2) {
            const typename L::Atom &a2 = sm.at[g2];
            const float *S2 = tail + g2 * T * 2 * KR;
            for (int q = lane; q < T * NR; q += 32) {
                const int bb = q / NR, n = q - bb * NR;
                const float x = a2.ab[n], y = a2.b[n];
                const float *sb = S2 + bb * 2 * KR;
                float *dst = accR + q * KR;  // = accR[b * NCR + n * KR]
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) dst[kk] += x * sb[kk] + y * sb[KR + kk];
            }
        }
        __syncwarp();

        // ---------------------------------------------------------------- angular coefficient gradient
        // per pair p (species b): X^b_nk += alpha_n f_k + beta_n f'_k with
        //   alpha_n = sum_lm dJ/dA_nlm Y_lm + dE/dA_nlm (grad Y_lm . p),
        //   beta_n  = (r^.lambda) sum_lm dE/dA_nlm Y_lm
        {
            float4 nxt = pair_or_zero(prs, sl, nAng);
            for (int c0 = 0; c0 < maxA; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxt;
                nxt = pair_or_zero(prs, k + SW, nAng);
                if (k < nAng) {
                    const int tj = pair_t(pd);
                    float lx, ly, lz;
                    pair_lambda(a, pd, fbx, fby, fbz, Wb, lx, ly, lz);
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    const float rinv = inv_norm(r2);
                    const float r = r2 * rinv;
                    const float ux = pd.x * rinv, uy = pd.y * rinv, uz = pd.z * rinv;
                    const float rl = ux * lx + uy * ly + uz * lz;
                    const float px = (lx - rl * ux) * rinv, py = (ly - rl * uy) * rinv, pz = (lz - rl * uz) * rinv;
                    float al[NA], be[NA];
#pragma unroll
                    for (int n = 0; n < NA; ++n) al[n] = be[n] = 0.0f;
                    ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                        const float ps = gx * px + gy * py + gz * pz;
                        const float4 *d4 = reinterpret_cast<const float4 *>(at.D + lm * NAP);
                        const float4 *h4 = reinterpret_cast<const float4 *>(at.Ah + lm * NAP);
#pragma unroll
                        for (int q = 0; q < NAP / 4; ++q) {
                            const float4 dq = d4[q], hq = h4[q];
                            const float dv[4] = {dq.x, dq.y, dq.z, dq.w}, hv[4] = {hq.x, hq.y, hq.z, hq.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int n = 4 * q + e;
                                if (n < NA) {
                                    al[n < NA ? n : 0] += dv[e] * Y + hv[e] * ps;
                                    be[n < NA ? n : 0] += hv[e] * Y;
                                }
                            }
                        }
                    });
                    float f[KA], fp[KA];
                    basis_val_der<KA>(r, a.inv_rcA, f, fp);
                    if (one_species) {
#pragma unroll
                        for (int n = 0; n < NA; ++n)
#pragma unroll
                            for (int kk = 0; kk < KA; ++kk)
                                X1[REG1 ? n * KA + kk : 0] += al[n] * f[kk] + (be[n] * rl) * fp[kk];
                    } else {
#pragma unroll
                        for (int n = 0; n < NA; ++n) sm.st.ab[grp][sl][n] = make_float2(al[n], be[n] * rl);
#pragma unroll
                        for (int kk = 0; kk < KA; ++kk) sm.st.ff[grp][sl][kk] = make_float2(f[kk], fp[kk]);
                        sm.st.t[grp][sl] = tj;
                    }
                }
                if (one_species) continue;
                __syncwarp();
                // every lane walks the rows of every atom of the batch (uniform control flow)
#pragma unroll 1
                for (int g2 = 0; g2 < G; ++g2) {
                    const int cnt = min(SW, __shfl_sync(FULL, nAng, g2 * SW) - c0);
#pragma unroll 2
                    for (int pp = 0; pp < cnt; ++pp) {
                        const int t = sm.st.t[g2][pp];
                        if (t != xb) {
                            close_tile();
                            xb = t;
                        }
                        if (tile_own) {
                            const float2 abv = sm.st.ab[g2][pp][tn];
#pragma unroll
                            for (int jj = 0; jj < TW; ++jj) {
                                if (tk0 + jj < KA) {
                                    const float2 ffv = sm.st.ff[g2][pp][tk0 + jj];
                                    X[jj] += abv.x * ffv.x + abv.y * ffv.y;
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
    __syncwarp();
    if (one_species && cur_t >= 0) flush_groups<V1, SW>(X1, accA, NCA, true, lane, true);
    close_tile();
    __syncwarp();
    if (cur_t >= 0) flush_slot(cur_t);
}

// ============================================================================= forward
// Three stages:
//   k_fwd_desc (per atom)  angular moments, radial descriptor, invariants -> q~, A;
//   k_net_fwd  (per chunk of atoms of one species, tiled products) the network (Eq. "ann"):
//                          h = tanh(W0 q~ - b0), E_i = w1.h - b1, b = s (W0^T (w1 (1 - h^2)));
//   k_fwd_pair (per atom)  dE_i/dA, the radial factors beta, pair gradients G_p, the
//                          atom's own force and virial sums.

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(128, VAR == 0 ? 4 : 5) k_fwd_desc(AtomArgs a) {
    grid_dep_wait();
    grid_dep_launch();
    using L = DescL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int G = L::G, NAP = L::NAP, NLMO = L::NLMO;
    constexpr int KR4 = round4(KR), KA4 = round4(KA);
    constexpr int VR = pow2ceil(KR);
    constexpr int VRN = pow2ceil(NR);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *Sr = base_ptr + sizeof(L) / sizeof(float) + grp * KR;  // [KR] of this group (one species)

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);
    const float *scale = a.par + po.scale;

    for (int bp = wbeg; bp < wend;) {
        const BatchAtom ba = load_batch<SW>(a, bp, wend, lane);
        const int ti = ba.ti, nb = ba.nb, i = ba.i;
        const bool act = grp < nb;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
        const float *cRi = a.par + po.cRp + (size_t)ti * T * NR * KR4;  // [b][n][KR4]
        const float *cAi = a.par + po.cAp + (size_t)ti * T * NA * KA4;  // [b][n][KA4]
        const int64_t beg = ba.beg;
        const int nRad = ba.nRad;
        const int nAng = ba.nAng;
        const int maxR = __reduce_max_sync(FULL, nRad);
        const int maxA = __reduce_max_sync(FULL, nAng);
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their pair records into L2
            const int4 nr = __ldg(a.rec + bp + grp);
            prefetch_l2(a.pair + nr.y, sizeof(float4) * (size_t)nr.z, sl, SW);
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
                float f[KA], g[NA];
                basis_val<KA>(r, a.inv_rcA, f);
                contract_c<NA, KA>(cAi + tj * NA * KA4, f, g);
                store_row4<NA>(sm.st.g[grp][sl], g);
                float Y[L3];
                ylm_val(pd.x * rinv, pd.y * rinv, pd.z * rinv, Y);
#pragma unroll
                for (int lm = 0; lm < L3; ++lm) sm.st.Y[grp][sl][lm] = Y[lm];
            }
            __syncwarp();
            const int cnt = min(SW, nAng - c0);
#pragma unroll 2
            for (int pp = 0; pp < cnt; ++pp) {
                float gv[NAP];
                load_row<NAP>(sm.st.g[grp][pp], gv);
#pragma unroll
                for (int j = 0; j < NLMO; ++j) {
                    const int lm = sl + j * SW;
                    if (lm < L3) {
                        const float y = sm.st.Y[grp][pp][lm];
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
            if (lm < L3) store_row4<NA>(at.A + lm * NAP, accA[j]);
        }

        // ---------------------------------------------------------------- radial descriptor q_n
        if (T == 1) {  // one species: S_k = sum_j f_k(r_ij), one reduction per atom, q = c S
            float v[VR];
#pragma unroll
            for (int k = 0; k < VR; ++k) v[k] = 0.0f;
            float4 nxr = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxr;
                nxr = pair_or_zero(prs, k + SW, nRad);
                if (k < nRad) {
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    float f[KR];
                    basis_val<KR>(r2 * inv_norm(r2), a.inv_rcR, f);
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) v[kk] += f[kk];
                }
            }
            for (int e = sl; e < KR; e += SW) Sr[e] = 0.0f;
            __syncwarp();
            if (__any_sync(FULL, nRad > 0)) flush_groups<VR, SW>(v, Sr, KR, nRad > 0, lane, false);
            __syncwarp();
            for (int n = sl; n < NR; n += SW) {
                float q = 0.0f;
                const float *cr = cRi + n * KR4;
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) q += __ldg(cr + kk) * Sr[kk];
                at.q[n] = q;
            }
        } else {  // several species: every lane adds g_n = sum_k c^{t_i t_j}_nk f_k of its own pairs
            float qv[VRN];
#pragma unroll
            for (int n = 0; n < VRN; ++n) qv[n] = 0.0f;
            float4 nxr = pair_or_zero(prs, sl, nRad);
            for (int c0 = 0; c0 < maxR; c0 += SW) {
                const int k = c0 + sl;
                const float4 pd = nxr;
                nxr = pair_or_zero(prs, k + SW, nRad);
                if (k < nRad) {
                    const float r2 = pd.x * pd.x + pd.y * pd.y + pd.z * pd.z;
                    float f[KR], g[NR];
                    basis_val<KR>(r2 * inv_norm(r2), a.inv_rcR, f);
                    contract_c<NR, KR>(cRi + pair_t(pd) * NR * KR4, f, g);
#pragma unroll
                    for (int n = 0; n < NR; ++n) qv[n] += g[n];
                }
            }
            for (int n = sl; n < NR; n += SW) at.q[n] = 0.0f;
            __syncwarp();
            if (__any_sync(FULL, nRad > 0)) flush_groups<VRN, SW>(qv, at.q, NR, nRad > 0, lane, false);
        }
        __syncwarp();

        // ---------------------------------------------------------------- invariants (Eq. "q3b", 4-/5-body)
        for (int e = sl; e < 4 * NA; e += SW) {
            const int n = e % NA, l = e / NA + 1;
            float s2 = 0.0f;
            for (int m = 0; m < 2 * l + 1; ++m) {
                const float v = at.A[(l * l - 1 + m) * NAP + n];
                s2 += v * v;
            }
            at.q[NR + (l - 1) * NA + n] = s2;
        }
        for (int n = sl; n < NA; n += SW) {
            float a2[5], Mt[6], M2[6];
            l2_block<NAP>(at.A, n, a2);
            l2_matrix(a2, Mt);
            sym_prod(Mt, Mt, M2);
            at.q[NR + 4 * NA + n] = KAPPA_REAL * sym_trace_prod(M2, Mt);
            const float x0 = at.A[n], x1 = at.A[NAP + n], x2 = at.A[2 * NAP + n];
            const float q1 = x0 * x0 + x1 * x1 + x2 * x2;
            at.q[NR + 5 * NA + n] = q1 * q1;
        }
        __syncwarp();
        if (act) {
            for (int e = sl; e < ND; e += SW) a.st_qt[(size_t)wi * ND + e] = at.q[e] * scale[e];
            for (int e = sl; e < L3 * NA; e += SW) {  // [lm][n], n packed
                const int lm = e / NA, n = e - lm * NA;
                a.st_A[(size_t)wi * NA * L3 + e] = at.A[lm * NAP + n];
            }
            if (a.q_raw)
                for (int e = sl; e < ND; e += SW) a.q_raw[(size_t)i * ND + e] = at.q[e];
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------- network forward
// Per chunk of <= 128 work positions of one species t, in tiles of 64 atoms (16 for chunks of
// at most 16) (Eq. "ann"):
//   h = tanh(W0 q~ - b0),  E = w1 . h - b1,  u = w1 (1 - h^2),  b = s (W0^T u).
// Same tiling as the network reverse pass.
template <class S, int RX>
__host__ __device__ inline size_t net_fwd_smem(int NN) {
    constexpr int R = 16 * RX;
    const size_t NDQ = round4(S::ND), NNP = round4(NN);
    return sizeof(float) * (NDQ * R + NNP * R + (size_t)S::ND * NNP + (size_t)NN * NDQ + R);
}

template <class S, int RX>
__global__ void __launch_bounds__(256) k_net_fwd(AtomArgs a) {
    constexpr int R = 16 * RX;  // tile rows: 16 row groups of RX
    grid_dep_wait();
    grid_dep_launch();
    constexpr int ND = S::ND, NDQ = round4(ND);
    extern __shared__ __align__(16) float smn[];
    const int NN = a.NN, NNP = round4(NN), T = a.T;
    float *Q = smn;                 // [NDQ][R] q~, transposed
    float *U = Q + NDQ * R;      // [NNP][R] u, transposed
    float *Wt = U + NNP * R;     // [ND][NNP]  W0^T of the species
    float *Wn = Wt + ND * NNP;      // [NN][NDQ]  W0 of the species
    float *Es = Wn + NN * NDQ;      // [R]     energies of the tile's atoms
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int rc0 = a.chunks[blockIdx.x], rc1 = a.chunks[blockIdx.x + 1];
    if (rc0 >= rc1) return;
    const int t = __ldg(a.rec2 + rc0).x;
    const ParOff po = par_offsets(T, NN, S::NR, S::KR, S::NA, S::KA);
    const float *W0 = a.par + po.w0 + (size_t)t * NN * ND;
    const float *W0T = a.par + po.w0t + (size_t)t * ND * NN;
    const float *b0 = a.par + po.b0 + (size_t)t * NN;
    const float *w1 = a.par + po.w1 + (size_t)t * NN;
    const float b1 = a.par[po.b1];
    const float *scale = a.par + po.scale;
    block_stage<256>(
        ND * NNP,
        [&](int e) {
            const int k = e / NNP, mu = e - k * NNP;
            return mu < NN ? __ldg(W0T + (size_t)k * NN + mu) : 0.0f;
        },
        [&](int e, float x) { Wt[e] = x; });
    block_stage<256>(
        NN * NDQ,
        [&](int e) {
            const int mu = e / NDQ, v = e - mu * NDQ;
            return v < ND ? __ldg(W0 + (size_t)mu * ND + v) : 0.0f;
        },
        [&](int e, float x) { Wn[e] = x; });
    for (int rb = rc0; rb < rc1; rb += R) {
        const int nr = min(R, rc1 - rb);
        __syncthreads();  // the weights are staged; the previous tile is done with Q, U, Es
        block_stage<256>(
            R * NDQ,
            [&](int e) {
                const int r = e / NDQ, k = e - r * NDQ;
                return (r < nr && k < ND) ? __ldg(a.st_qt + (size_t)(rb + r) * ND + k) : 0.0f;
            },
            [&](int e, float x) {
                const int r = e / NDQ, k = e - r * NDQ;
                Q[k * R + r] = x;
            });
        if (threadIdx.x < R) Es[threadIdx.x] = 0.0f;
        __syncthreads();
        const int r0 = ty * RX;
        for (int cb = 0; cb < NNP; cb += 64) {
            const int mu0 = cb + tx * 4;
            float ep[RX];
#pragma unroll
            for (int x = 0; x < RX; ++x) ep[x] = 0.0f;  // w1 . h over this thread's 4 neurons
            if (mu0 < NNP) {
                float acc[RX][4];
#pragma unroll
                for (int x = 0; x < RX; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
#pragma unroll 7
                for (int k = 0; k < ND; ++k) {
                    float q[RX];
                    ld_rows<RX>(Q + k * R + r0, q);
                    const float4 w4 = *reinterpret_cast<const float4 *>(Wt + k * NNP + mu0);
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < RX; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] += q[x] * wv[y];
                }
#pragma unroll
                for (int x = 0; x < RX; ++x) {
                    const int r = r0 + x;
                    const bool row = r < nr;
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int mu = mu0 + y;
                        float uu = 0.0f;
                        if (row && mu < NN) {
                            const float h = tanhf(acc[x][y] - b0[mu]);
                            const float wo = w1[mu];
                            a.st_h[(size_t)(rb + r) * NN + mu] = h;
                            ep[x] += wo * h;
                            uu = wo * (1.0f - h * h);
                        }
                        U[mu * R + r] = uu;
                    }
                }
            }
            // energies: the 16 column threads of a row group add their neuron sums in a fixed order
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                float v = ep[x];
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                if (tx == 0) Es[r0 + x] += v;
            }
        }
        __syncthreads();
        if (threadIdx.x < nr) a.st_E[rb + threadIdx.x] = Es[threadIdx.x] - b1;
        for (int cb = 0; cb < NDQ; cb += 64) {
            const int v0 = cb + tx * 4;
            if (v0 < NDQ) {
                float ab[RX][4];
#pragma unroll
                for (int x = 0; x < RX; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) ab[x][y] = 0.0f;
#pragma unroll 5
                for (int mu = 0; mu < NN; ++mu) {
                    float uu[RX];
                    ld_rows<RX>(U + mu * R + r0, uu);
                    const float4 w4 = *reinterpret_cast<const float4 *>(Wn + mu * NDQ + v0);
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < RX; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) ab[x][y] += uu[x] * wv[y];
                }
#pragma unroll
                for (int x = 0; x < RX; ++x) {
                    const int r = r0 + x;
                    if (r < nr) {
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const int v = v0 + y;
                            if (v < ND) a.st_b[(size_t)(rb + r) * ND + v] = ab[x][y] * scale[v];
                        }
                    }
                }
            }
        }
    }
}

template <class S, int SW, int VAR>
__global__ void __launch_bounds__(128, VAR == 0 ? 4 : 5) k_fwd_pair(AtomArgs a) {
    grid_dep_wait();
    grid_dep_launch();
    using L = PairL<S, SW>;
    constexpr int NR = S::NR, KR = S::KR, NA = S::NA, KA = S::KA, ND = S::ND;
    constexpr int G = L::G, NAP = L::NAP, NLMO = L::NLMO;
    constexpr int KR4 = round4(KR), KA4 = round4(KA);
    extern __shared__ __align__(16) float smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / SW, sl = lane % SW;
    const int T = a.T, NN = a.NN;
    float *base_ptr = smem_raw + wib * (L::bytes(T, NN) / sizeof(float));
    L &sm = *reinterpret_cast<L *>(base_ptr);
    float *beta = base_ptr + sizeof(L) / sizeof(float) + grp * T * KR;  // [T][KR] of this group

    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    const int wbeg = a.warp_begin[w], wend = a.warp_begin[w + 1];
    const ParOff po = par_offsets(T, NN, NR, KR, NA, KA);

    for (int bp = wbeg; bp < wend;) {
        const BatchAtom ba = load_batch<SW>(a, bp, wend, lane);
        const int ti = ba.ti, nb = ba.nb, i = ba.i;
        const bool act = grp < nb;
        const int wi = bp + (act ? grp : 0);
        bp += nb;
        const float *cRi = a.par + po.cRp + (size_t)ti * T * NR * KR4;
        const float *cAi = a.par + po.cAp + (size_t)ti * T * NA * KA4;
        const int64_t beg = ba.beg;
        const int nRad = ba.nRad;
        const int nAng = ba.nAng;
        typename L::Atom &at = sm.at[grp];
        if (bp + grp < wend) {  // the atoms after this batch: bring their pair records into L2
            const int4 nr = __ldg(a.rec + bp + grp);
            prefetch_l2(a.pair + nr.y, sizeof(float4) * (size_t)nr.z, sl, SW);
        }
        load_lm_rows<NA, NAP, SW>(a.st_A + (size_t)wi * NA * L3, at.A, sl);
        gather_rows<ND, SW>(a.st_b + (size_t)wi * ND, sl, [&](int v, float x) { at.b[v] = x; });
        __syncwarp();

        // ---------------------------------------------------------------- dE_i/dA and radial factors
        for (int n = sl; n < NA; n += SW) {
            float a2[5], Mt[6], M2[6], pr[5];
            l2_block<NAP>(at.A, n, a2);
            l2_matrix(a2, Mt);
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
                float ah[NA];
#pragma unroll
                for (int n = 0; n < NA; ++n) {
                    const float av = at.A[lm * NAP + n];
                    float x = 2.0f * at.b[NR + (l - 1) * NA + n] * av;
                    if (l == 2) x += at.b[NR + 4 * NA + n] * at.G4[n * 5 + (lm - 3)];
                    if (l == 1) {
                        const float x0 = at.A[n], x1 = at.A[NAP + n], x2 = at.A[2 * NAP + n];
                        x += at.b[NR + 5 * NA + n] * 4.0f * (x0 * x0 + x1 * x1 + x2 * x2) * av;
                    }
                    ah[n] = x;
                }
                store_row4<NA>(at.Ah + lm * NAP, ah);
            }
        }
        for (int e = sl; e < T * KR; e += SW) {
            const int bb = e / KR, kk = e - bb * KR;
            float s2 = 0.0f;
#pragma unroll
            for (int n = 0; n < NR; ++n) s2 += at.b[n] * __ldg(cRi + (bb * NR + n) * KR4 + kk);
            beta[e] = s2;
        }
        __syncwarp();

        // ---------------------------------------------------------------- pair gradients
        const float4 *prs = a.pair + beg;
        const float *zbl_ti = a.zbl ? a.zbl + (size_t)ti * T * 2 : nullptr;
        float Ez = 0.0f;  // ZBL energy of this lane's pairs (half of each pair term)
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
            float f[KA], fp[KA], g[NA], gp[NA];
            basis_val_der<KA>(r, a.inv_rcA, f, fp);
            contract_c2<NA, KA>(cAi + tj * NA * KA4, f, fp, g, gp);
            float srad = 0.0f, Vx = 0.0f, Vy = 0.0f, Vz = 0.0f;
            ylm_each(ux, uy, uz, [&](int lm, float Y, float gx, float gy, float gz) {
                const float4 *h4 = reinterpret_cast<const float4 *>(at.Ah + lm * NAP);
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int q = 0; q < NAP / 4; ++q) {
                    const float4 h = h4[q];
                    const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (4 * q + e < NA) {
                            a1 += hv[e] * at_k<NA>(g, 4 * q + e);
                            a2 += hv[e] * at_k<NA>(gp, 4 * q + e);
                        }
                    }
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
            if (r < a.zbl_r2) {
                float ez, dez;
                zbl_term(r, zbl_ti[2 * tj], zbl_ti[2 * tj + 1], a.zbl_r1, a.zbl_r2, ez, dez);
                Ez += 0.5f * ez;
                srad += 0.5f * dez;
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
            if (r2 * rinv < a.zbl_r2) {
                float ez, dez;
                zbl_term(r2 * rinv, zbl_ti[2 * tj], zbl_ti[2 * tj + 1], a.zbl_r1, a.zbl_r2, ez, dez);
                Ez += 0.5f * ez;
                s2 += 0.5f * dez;
            }
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
            const float Ei = a.st_E[wi];
            float v[16] = {Fx, Fy, Fz, W9[0], W9[1], W9[2], W9[3], W9[4], W9[5], W9[6], W9[7], W9[8],
                           Ez, 0.0f, 0.0f, 0.0f};
            group_reduce_scatter<16, SW>(v, lane);
            const int base = grs_base<16, SW>(lane);
            if (act && (lane & GRS<16, SW>::DUP_MASK) == 0) {
#pragma unroll
                for (int o = 0; o < GRS<16, SW>::OUT; ++o) {
                    const int idx = base + o;
                    if (idx < 3) a.F_own[(size_t)i * 3 + idx] = v[o];
                    else if (idx < 12) a.W_atom[(size_t)i * 9 + idx - 3] = v[o];
                    else if (idx == 12) a.E_atom[i] = Ei + v[o];
                }
            }
        }
        __syncwarp();
    }
}

// ============================================================================= dispatch

// Forward stages: 0 = descriptors, 1 = network, 2 = pair gradients, -1 = all three.
template <class S, int SW, int VAR>
void launch_fwd_t(const AtomArgs &a, int blocks, int wpb, int stage, cudaStream_t st, bool pdl) {
    if (stage < 0 || stage == 0)
        launch_k(pdl, k_fwd_desc<S, SW, VAR>, blocks, wpb * 32, DescL<S, SW>::bytes(a.T, a.NN) * wpb, st, a);
    if ((stage < 0 || stage == 1) && a.n_chunks > 0) {  // 16-row tiles for chunks of at most 16
        if (a.chunk_rows <= 16) launch_k(pdl, k_net_fwd<S, 1>, a.n_chunks, 256, net_fwd_smem<S, 1>(a.NN), st, a);
        else launch_k(pdl, k_net_fwd<S, 4>, a.n_chunks, 256, net_fwd_smem<S, 4>(a.NN), st, a);
    }
    if (stage < 0 || stage == 2)
        launch_k(pdl, k_fwd_pair<S, SW, VAR>, blocks, wpb * 32, PairL<S, SW>::bytes(a.T, a.NN) * wpb, st, a);
}
// Adjoint stages: 0 = JVP, 1 = network reverse, 2 = coefficient gradient, -1 = all three.
template <class S, int SW, int VAR>
void launch_adj_t(const AtomArgs &a, int blocks, int wpb, int stage, cudaStream_t st, bool pdl) {
    if (stage < 0 || stage == 0)
        launch_k(pdl, k_adj_jvp<S, SW, VAR>, blocks, wpb * 32, JvpL<S, SW>::bytes(a.T, a.NN) * wpb, st, a);
    if ((stage < 0 || stage == 1) && a.n_chunks > 0) {
        if (a.chunk_rows <= 16) launch_k(pdl, k_net_rev<S, 1>, a.n_chunks, 256, net_rev_smem<S, 1>(a.NN), st, a);
        else launch_k(pdl, k_net_rev<S, 4>, a.n_chunks, 256, net_rev_smem<S, 4>(a.NN), st, a);
    }
    if (stage < 0 || stage == 2)
        launch_k(pdl, k_adj_cg<S, SW, VAR>, blocks, wpb * 32, CgL<S, SW>::bytes(a.T, a.NN) * wpb, st, a);
}
// per-warp shared memory of the larger of the two per-atom forward stages
template <class S, int SW>
size_t fwd_bytes_t(int T, int NN) {
    const size_t d = DescL<S, SW>::bytes(T, NN), p = PairL<S, SW>::bytes(T, NN);
    return d > p ? d : p;
}
// per-warp shared memory of the larger of the two per-atom adjoint stages
template <class S, int SW>
size_t adj_bytes_t(int T, int NN) {
    const size_t j = JvpL<S, SW>::bytes(T, NN), c = CgL<S, SW>::bytes(T, NN);
    return j > c ? j : c;
}

// Variant v: SW = 8 (v < 2), 16 (v < 4) or 32, register budget VAR = v & 1 (blocks of at most 128 threads;
// 0: four blocks per SM, 128 registers; 1: five blocks per SM, 96 registers).
template <int NR, int KR, int NA, int KA>
KernelSet make_set() {
    using S = Shape<NR, KR, NA, KA>;
    KernelSet k;
    k.NR = NR;
    k.KR = KR;
    k.NA = NA;
    k.KA = KA;
    k.fwd_fn[0] = (const void *)k_fwd_pair<S, 8, 0>;
    k.fwd_fn[1] = (const void *)k_fwd_pair<S, 8, 1>;
    k.fwd_fn[2] = (const void *)k_fwd_pair<S, 16, 0>;
    k.fwd_fn[3] = (const void *)k_fwd_pair<S, 16, 1>;
    k.fwd_fn[4] = (const void *)k_fwd_pair<S, 32, 0>;
    k.fwd_fn[5] = (const void *)k_fwd_pair<S, 32, 1>;
    k.desc_fn[0] = (const void *)k_fwd_desc<S, 8, 0>;
    k.desc_fn[1] = (const void *)k_fwd_desc<S, 8, 1>;
    k.desc_fn[2] = (const void *)k_fwd_desc<S, 16, 0>;
    k.desc_fn[3] = (const void *)k_fwd_desc<S, 16, 1>;
    k.desc_fn[4] = (const void *)k_fwd_desc<S, 32, 0>;
    k.desc_fn[5] = (const void *)k_fwd_desc<S, 32, 1>;
    k.net_fwd_fn[0] = (const void *)k_net_fwd<S, 4>;
    k.net_fwd_fn[1] = (const void *)k_net_fwd<S, 1>;
    k.net_fwd_smem = net_fwd_smem<S, 4>;
    k.adj_fn[0] = (const void *)k_adj_cg<S, 8, 0>;
    k.adj_fn[1] = (const void *)k_adj_cg<S, 8, 1>;
    k.adj_fn[2] = (const void *)k_adj_cg<S, 16, 0>;
    k.adj_fn[3] = (const void *)k_adj_cg<S, 16, 1>;
    k.adj_fn[4] = (const void *)k_adj_cg<S, 32, 0>;
    k.adj_fn[5] = (const void *)k_adj_cg<S, 32, 1>;
    k.jvp_fn[0] = (const void *)k_adj_jvp<S, 8, 0>;
    k.jvp_fn[1] = (const void *)k_adj_jvp<S, 8, 1>;
    k.jvp_fn[2] = (const void *)k_adj_jvp<S, 16, 0>;
    k.jvp_fn[3] = (const void *)k_adj_jvp<S, 16, 1>;
    k.jvp_fn[4] = (const void *)k_adj_jvp<S, 32, 0>;
    k.jvp_fn[5] = (const void *)k_adj_jvp<S, 32, 1>;
    k.net_rev_fn[0] = (const void *)k_net_rev<S, 4>;
    k.net_rev_fn[1] = (const void *)k_net_rev<S, 1>;
    k.net_rev_smem = net_rev_smem<S, 4>;
    k.launch_fwd[0] = launch_fwd_t<S, 8, 0>;
    k.launch_fwd[1] = launch_fwd_t<S, 8, 1>;
    k.launch_fwd[2] = launch_fwd_t<S, 16, 0>;
    k.launch_fwd[3] = launch_fwd_t<S, 16, 1>;
    k.launch_fwd[4] = launch_fwd_t<S, 32, 0>;
    k.launch_fwd[5] = launch_fwd_t<S, 32, 1>;
    k.launch_adj[0] = launch_adj_t<S, 8, 0>;
    k.launch_adj[1] = launch_adj_t<S, 8, 1>;
    k.launch_adj[2] = launch_adj_t<S, 16, 0>;
    k.launch_adj[3] = launch_adj_t<S, 16, 1>;
    k.launch_adj[4] = launch_adj_t<S, 32, 0>;
    k.launch_adj[5] = launch_adj_t<S, 32, 1>;
    k.fwd_smem[0] = k.fwd_smem[1] = fwd_bytes_t<S, 8>;
    k.fwd_smem[2] = k.fwd_smem[3] = fwd_bytes_t<S, 16>;
    k.fwd_smem[4] = k.fwd_smem[5] = fwd_bytes_t<S, 32>;
    k.adj_smem[0] = k.adj_smem[1] = adj_bytes_t<S, 8>;
    k.adj_smem[2] = k.adj_smem[3] = adj_bytes_t<S, 16>;
    k.adj_smem[4] = k.adj_smem[5] = adj_bytes_t<S, 32>;
    for (int v = 0; v < NVAR; ++v) {
        k.max_wpb[v] = 4;
        k.sw[v] = v < 2 ? 8 : v < 4 ? 16 : 32;
    }
    return k;
}

}  // namespace nep
