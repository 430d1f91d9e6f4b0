// Internal definitions shared by the CUDA translation units of the NEP library.
//
// Padded internal layout.  The per-atom kernels are compiled for a shape bucket
// (NR, KR, NA, KA) = compile-time upper bounds of N_R = n_max_R + 1, K_R =
// basis_R + 1, N_A, K_A.  Parameters are expanded into a padded buffer where the
// unused radial/angular channels and basis functions carry zero coefficients and
// the unused descriptor components carry zero scale and zero weights, so every
// loop runs to a compile-time bound without masks.  The padded descriptor order
// is [q_n (NR) | q_nl l = 1..4 (NA each) | q4_n (NA) | q5_n (NA)]: ND = NR + 6 NA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nep {

constexpr unsigned FULL = 0xffffffffu;
constexpr int L3 = 24;        // sum_{l=1..4} (2l+1)
constexpr int TMAX = 16;      // species limit
constexpr int NNMAX = 128;    // hidden-neuron limit
constexpr float PI_F = 3.14159265358979323846f;

template <int NR_, int KR_, int NA_, int KA_>
struct Shape {
    static constexpr int NR = NR_, KR = KR_, NA = NA_, KA = KA_;
    static constexpr int ND = NR + 6 * NA;
    static constexpr int NCR = NR * KR;
    static constexpr int NCA = NA * KA;
    static constexpr int NC = NCR + NCA;
};

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

// Offsets (in floats) of the padded parameter buffer.  cRp / cAp repeat the coefficients
// with each (n) row padded to a multiple of 4 floats and 16-byte aligned, for float4 loads.
struct ParOff {
    int64_t w0, w0t, b0, w1, b1, cR, cA, scale, cRp, cAp, total;
};

__host__ __device__ inline ParOff par_offsets(int T, int NN, int NR, int KR, int NA, int KA) {
    ParOff o;
    const int64_t ND = NR + 6 * NA;
    o.w0 = 0;                                  // [T][NN][ND]
    o.w0t = o.w0 + (int64_t)T * NN * ND;       // [T][ND][NN]
    o.b0 = o.w0t + (int64_t)T * NN * ND;       // [T][NN]
    o.w1 = o.b0 + (int64_t)T * NN;             // [T][NN]
    o.b1 = o.w1 + (int64_t)T * NN;             // [1] (+3 pad)
    o.cR = o.b1 + 4;                           // [T][T][NR][KR]
    o.cA = o.cR + (int64_t)T * T * NR * KR;    // [T][T][NA][KA]
    o.scale = o.cA + (int64_t)T * T * NA * KA; // [ND]
    o.cRp = (o.scale + ND + 3) & ~(int64_t)3;  // [T][T][NR][round4(KR)]
    o.cAp = o.cRp + (int64_t)T * T * NR * round4(KR);  // [T][T][NA][round4(KA)]
    o.total = o.cAp + (int64_t)T * T * NA * round4(KA);
    return o;
}

// Runtime arguments of the per-atom kernels.
struct AtomArgs {
    // schedule
    const int *work;        // [Na] atom index at each work position (atoms sorted by species)
    const int4 *rec;        // [Na] per work position: atom i, first pair, radial and angular pair counts
    const int2 *rec2;       // [Na] per work position: species and structure of the atom
    const int *warp_begin;  // [W+1] work-position range of each warp
    // geometry (cached by the neighbour build)
    const int64_t *nbr_off; // [Na+1]
    const int *n_ang;       // [Na] angular neighbours (the first entries of each list)
    const float4 *pair;     // [M] (dx, dy, dz, bits(j << 4 | t_j))
    const int *type;        // [Na]
    const int *struct_of;   // [Na]
    // model
    const float *par;       // padded parameters (ParOff layout)
    int T, NN;
    float inv_rcR, inv_rcA, rc2A;
    const float *zbl;       // [T][T][2]: e^2/(4 pi eps0) Z_i Z_j and 1/a_ij of the ZBL term
    float zbl_r1, zbl_r2;   // ZBL switch radii (zbl_r2 = 0: no ZBL term)
    // forward outputs
    float *E_atom;          // [Na]
    float *F_own;           // [Na*3]   sum over own pairs of G
    float *W_atom;          // [Na*9]
    float4 *G;              // [M] pair gradients dE_i/dd_p
    float *st_qt;           // [Na_work][ND] normalised descriptors (by work position)
    float *st_h;            // [Na_work][NN] hidden activations
    float *st_A;            // [Na_work][NA*24] angular moments
    // adjoint inputs
    const float4 *fbar;     // [Na]    dL/dF (x, y, z, unused)
    const float *ebar;      // [Ns]    dL/dE_s
    const float *wbar;      // [Ns*9]  dL/dW_s
    // adjoint outputs
    float *zt, *ut, *om;    // [Na_work][NN]
    float *dqt;             // [Na_work][ND] normalised descriptor JVP
    float *cpart;           // [(W + T)][T][NC] per-warp c-gradient partials
    float *q_raw;           // optional [Na][ND] raw descriptors (descriptor export), may be null
    // adjoint stages: JVP -> network reverse (chunks of <= 128 work positions of one
    // species) -> coefficient gradient
    const int *chunks;      // [n_chunks + 1] chunk boundaries (work positions)
    int n_chunks;
    int chunk_rows;         // the longest chunk (<= 16: the network kernels take 16-row tiles)
    int NDP;                // padded descriptor length
    float *st_D;            // [Na_work][NA*24] JVP of the angular moments, [lm][n]
    float *st_S;            // [Na_work][T][2 KR] radial species sums S^b_k | S'^b_k
    float *st_b;            // [Na_work][ND] s * dE_i/dq~
    float *st_ab;           // [Na_work][ND] abar = dJ/dq (scaled)
    float *st_E;            // [Na_work] network energy of each atom (without the ZBL term)
};



// ----------------------------------------------------------------------------- warp helpers

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Programmatic dependent launch.  Every kernel of the step calls grid_dep_wait() before
// its first global-memory access: it returns once the kernel launched before it in the
// stream has completed and its writes are visible (at once when launched without the
// attribute).  grid_dep_launch() lets the next kernel's blocks be scheduled early; they
// wait in grid_dep_wait(), so only launch latency overlaps, never memory traffic.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch of a kernel that starts with grid_dep_wait(); pdl allows it to be scheduled while
// the previous kernel of the stream drains (also inside a captured graph).
template <typename... P, typename... A>
inline cudaError_t launch_k(bool pdl, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<A &&>(args)...);
}

// Transposing warp reduction of V values per lane (V a power of two).  Recursive
// halving: at each step a lane keeps one half of its values and adds the half
// its partner kept.  After min(log2 V, 5) steps lane l holds V/32 fully reduced
// values (or one value, completed by butterfly steps, when V < 32) whose
// original indices are base(l) + 0, 1, ...  Fixed pairing: deterministic.
template <int V>
struct RS {
    static constexpr int STEPS = (V >= 32) ? 5 : (V == 16 ? 4 : V == 8 ? 3 : V == 4 ? 2 : V == 2 ? 1 : 0);
    static constexpr int OUT = (V >= 32) ? V / 32 : 1;
    // lanes that hold duplicate copies differ in their low (5 - STEPS) bits
    static constexpr int DUP_MASK = (1 << (5 - STEPS)) - 1;
};

template <int V>
__device__ __forceinline__ int rs_base(int lane) {
    int base = 0;
    int h = V / 2;
    int o = 16;
#pragma unroll
    for (int s = 0; s < RS<V>::STEPS; ++s) {
        if (lane & o) base += h;
        h >>= 1;
        o >>= 1;
    }
    return base;
}

template <int V>
__device__ __forceinline__ void reduce_scatter(float *v, int lane) {
    int o = 16;
#pragma unroll
    for (int h = V / 2, s = 0; s < RS<V>::STEPS; h >>= 1, ++s) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, o);
        }
        o >>= 1;
    }
#pragma unroll
    for (int s = RS<V>::STEPS; s < 5; ++s) {
        v[0] += __shfl_xor_sync(FULL, v[0], o);
        o >>= 1;
    }
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Group versions: a group is SW consecutive lanes (SW = 8, 16 or 32) aligned to SW.
// XOR shuffles with offsets below SW stay inside the group.
template <int V, int SW>
struct GRS {
    static constexpr int LSW = ilog2(SW);
    static constexpr int LV = ilog2(V);
    static constexpr int STEPS = LV < LSW ? LV : LSW;
    static constexpr int OUT = V >= SW ? V / SW : 1;
    static constexpr int DUP_MASK = (1 << (LSW - STEPS)) - 1;
};

template <int V, int SW>
__device__ __forceinline__ int grs_base(int lane) {
    int base = 0, h = V / 2, o = SW / 2;
#pragma unroll
    for (int s = 0; s < GRS<V, SW>::STEPS; ++s) {
        if (lane & o) base += h;
        h >>= 1;
        o >>= 1;
    }
    return base;
}

// Transposing reduction of V values over the SW lanes of each group (fixed pairing).
template <int V, int SW>
__device__ __forceinline__ void group_reduce_scatter(float *v, int lane) {
    int o = SW / 2;
#pragma unroll
    for (int h = V / 2, s = 0; s < GRS<V, SW>::STEPS; h >>= 1, ++s) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, o);
        }
        o >>= 1;
    }
#pragma unroll
    for (int s = GRS<V, SW>::STEPS; s < GRS<V, SW>::LSW; ++s) {
        v[0] += __shfl_xor_sync(FULL, v[0], o);
        o >>= 1;
    }
}

template <int SW>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = SW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int SW>
__device__ __forceinline__ unsigned group_bits(unsigned ballot, int lane) {
    if (SW == 32) return ballot;
    return (ballot >> (lane & ~(SW - 1))) & ((1u << SW) - 1u);
}

__host__ __device__ constexpr int pow2ceil(int v) {
    return v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : v <= 8 ? 8 : v <= 16 ? 16 : v <= 32 ? 32 : v <= 64 ? 64 : v <= 128 ? 128 : 256;
}

// ----------------------------------------------------------------------------- basis functions
// f_k(r) = 1/2 (T_k(x) + 1) f_c(r), x = 2 (r/rc - 1)^2 - 1, f_c = 1/2 (cos(pi r/rc) + 1)
// (Methods, "NEP descriptors"); derivatives by the Chebyshev recurrences
// T_{k+1} = 2x T_k - T_{k-1},  T'_{k+1} = 2 T_k + 2x T'_k - T'_{k-1}.
// Only called for pairs with r < rc.

// The cutoff uses the hardware sine/cosine (absolute error about 2^-21 on [-pi, pi]);
// f_c only multiplies the basis, so this stays far inside the FP32 path's tolerance.
template <int K>
__device__ __forceinline__ void basis_val(float r, float inv_rc, float *f) {
    const float u = r * inv_rc;
    const float fc = 0.5f * __cosf(PI_F * u) + 0.5f;
    const float y = u - 1.0f;
    const float x = 2.0f * y * y - 1.0f;
    float tm1 = 1.0f, t = x;
    f[0] = fc;
    if (K > 1) f[1] = 0.5f * (x + 1.0f) * fc;
#pragma unroll
    for (int k = 2; k < K; ++k) {
        const float tn = 2.0f * x * t - tm1;
        tm1 = t;
        t = tn;
        f[k] = 0.5f * (tn + 1.0f) * fc;
    }
}

template <int K>
__device__ __forceinline__ void basis_val_der(float r, float inv_rc, float *f, float *fp) {
    const float u = r * inv_rc;
    float s, c;
    __sincosf(PI_F * u, &s, &c);
    const float fc = 0.5f * c + 0.5f;
    const float dfc = -0.5f * PI_F * inv_rc * s;
    const float y = u - 1.0f;
    const float x = 2.0f * y * y - 1.0f;
    const float dxdr = 4.0f * y * inv_rc;
    float tm1 = 1.0f, t = x, dm1 = 0.0f, dt = 1.0f;
    f[0] = fc;
    fp[0] = dfc;
    if (K > 1) {
        f[1] = 0.5f * (x + 1.0f) * fc;
        fp[1] = 0.5f * (dxdr * fc + (x + 1.0f) * dfc);
    }
#pragma unroll
    for (int k = 2; k < K; ++k) {
        const float tn = 2.0f * x * t - tm1;
        const float dn = 2.0f * t + 2.0f * x * dt - dm1;
        tm1 = t;
        t = tn;
        dm1 = dt;
        dt = dn;
        f[k] = 0.5f * (tn + 1.0f) * fc;
        fp[k] = 0.5f * (dn * dxdr * fc + (tn + 1.0f) * dfc);
    }
}

// ----------------------------------------------------------------------------- real harmonics
// Orthonormal real spherical harmonics of a unit vector (x, y, z), l = 1..4, written
// as polynomials P_lm(x, y, z) that equal Y_lm on the unit sphere, stored at index
// (l*l - 1) + (m + l), m = -l..l.  The gradient of Y_lm(d/|d|) with respect to d is
// (I - u u^T) grad P_lm(u) / |d|, so any extension off the sphere may be used.
// Optional gradient outputs gx, gy, gz (grad P_lm).

struct YlmC {
    static constexpr float c1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
    static constexpr float c2a = 1.09254843059207918f;  // sqrt(15/pi)/2
    static constexpr float c2b = 0.31539156525252005f;  // sqrt(5/pi)/4
    static constexpr float c2c = 0.54627421529603959f;  // sqrt(15/pi)/4
    static constexpr float c3a = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
    static constexpr float c3b = 2.89061144264055381f;  // sqrt(105/pi)/2
    static constexpr float c3c = 0.45704579946446577f;  // sqrt(21/(2 pi))/4
    static constexpr float c3d = 0.37317633259011540f;  // sqrt(7/pi)/4
    static constexpr float c3e = 1.44530572132027690f;  // sqrt(105/pi)/4
    static constexpr float c4a = 2.50334294179670458f;  // 3 sqrt(35/pi)/4
    static constexpr float c4b = 1.77013076977993045f;  // 3 sqrt(35/(2 pi))/4
    static constexpr float c4c = 0.94617469575756008f;  // 3 sqrt(5/pi)/4
    static constexpr float c4d = 0.66904654355728921f;  // 3 sqrt(5/(2 pi))/4
    static constexpr float c4e = 0.10578554691520431f;  // 3/(16 sqrt(pi))
    static constexpr float c4f = 0.47308734787878004f;  // 3 sqrt(5/pi)/8
    static constexpr float c4g = 0.62583573544917614f;  // 3 sqrt(35/pi)/16
};

__device__ __forceinline__ void ylm_val(float x, float y, float z, float *Y) {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    Y[0] = YlmC::c1 * y;
    Y[1] = YlmC::c1 * z;
    Y[2] = YlmC::c1 * x;
    Y[3] = YlmC::c2a * x * y;
    Y[4] = YlmC::c2a * y * z;
    Y[5] = YlmC::c2b * (3.0f * z2 - 1.0f);
    Y[6] = YlmC::c2a * x * z;
    Y[7] = YlmC::c2c * (x2 - y2);
    Y[8] = YlmC::c3a * y * (3.0f * x2 - y2);
    Y[9] = YlmC::c3b * x * y * z;
    Y[10] = YlmC::c3c * y * (5.0f * z2 - 1.0f);
    Y[11] = YlmC::c3d * z * (5.0f * z2 - 3.0f);
    Y[12] = YlmC::c3c * x * (5.0f * z2 - 1.0f);
    Y[13] = YlmC::c3e * z * (x2 - y2);
    Y[14] = YlmC::c3a * x * (x2 - 3.0f * y2);
    Y[15] = YlmC::c4a * x * y * (x2 - y2);
    Y[16] = YlmC::c4b * y * z * (3.0f * x2 - y2);
    Y[17] = YlmC::c4c * x * y * (7.0f * z2 - 1.0f);
    Y[18] = YlmC::c4d * y * z * (7.0f * z2 - 3.0f);
    Y[19] = YlmC::c4e * ((35.0f * z2 - 30.0f) * z2 + 3.0f);
    Y[20] = YlmC::c4d * x * z * (7.0f * z2 - 3.0f);
    Y[21] = YlmC::c4f * (x2 - y2) * (7.0f * z2 - 1.0f);
    Y[22] = YlmC::c4b * x * z * (x2 - 3.0f * y2);
    Y[23] = YlmC::c4g * (x2 * (x2 - 3.0f * y2) - y2 * (3.0f * x2 - y2));
}

__device__ __forceinline__ void ylm_grad(float x, float y, float z, float *gx, float *gy, float *gz) {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    // l = 1
    gx[0] = 0.0f;            gy[0] = YlmC::c1;        gz[0] = 0.0f;
    gx[1] = 0.0f;            gy[1] = 0.0f;            gz[1] = YlmC::c1;
    gx[2] = YlmC::c1;        gy[2] = 0.0f;            gz[2] = 0.0f;
    // l = 2
    gx[3] = YlmC::c2a * y;   gy[3] = YlmC::c2a * x;   gz[3] = 0.0f;
    gx[4] = 0.0f;            gy[4] = YlmC::c2a * z;   gz[4] = YlmC::c2a * y;
    gx[5] = 0.0f;            gy[5] = 0.0f;            gz[5] = YlmC::c2b * 6.0f * z;
    gx[6] = YlmC::c2a * z;   gy[6] = 0.0f;            gz[6] = YlmC::c2a * x;
    gx[7] = YlmC::c2c * 2.0f * x; gy[7] = -YlmC::c2c * 2.0f * y; gz[7] = 0.0f;
    // l = 3
    gx[8] = YlmC::c3a * 6.0f * x * y;
    gy[8] = YlmC::c3a * 3.0f * (x2 - y2);
    gz[8] = 0.0f;
    gx[9] = YlmC::c3b * y * z;
    gy[9] = YlmC::c3b * x * z;
    gz[9] = YlmC::c3b * x * y;
    gx[10] = 0.0f;
    gy[10] = YlmC::c3c * (5.0f * z2 - 1.0f);
    gz[10] = YlmC::c3c * 10.0f * y * z;
    gx[11] = 0.0f;
    gy[11] = 0.0f;
    gz[11] = YlmC::c3d * (15.0f * z2 - 3.0f);
    gx[12] = YlmC::c3c * (5.0f * z2 - 1.0f);
    gy[12] = 0.0f;
    gz[12] = YlmC::c3c * 10.0f * x * z;
    gx[13] = YlmC::c3e * 2.0f * x * z;
    gy[13] = -YlmC::c3e * 2.0f * y * z;
    gz[13] = YlmC::c3e * (x2 - y2);
    gx[14] = YlmC::c3a * 3.0f * (x2 - y2);
    gy[14] = -YlmC::c3a * 6.0f * x * y;
    gz[14] = 0.0f;
    // l = 4
    gx[15] = YlmC::c4a * y * (3.0f * x2 - y2);
    gy[15] = YlmC::c4a * x * (x2 - 3.0f * y2);
    gz[15] = 0.0f;
    gx[16] = YlmC::c4b * 6.0f * x * y * z;
    gy[16] = YlmC::c4b * 3.0f * z * (x2 - y2);
    gz[16] = YlmC::c4b * y * (3.0f * x2 - y2);
    gx[17] = YlmC::c4c * y * (7.0f * z2 - 1.0f);
    gy[17] = YlmC::c4c * x * (7.0f * z2 - 1.0f);
    gz[17] = YlmC::c4c * 14.0f * x * y * z;
    gx[18] = 0.0f;
    gy[18] = YlmC::c4d * z * (7.0f * z2 - 3.0f);
    gz[18] = YlmC::c4d * y * (21.0f * z2 - 3.0f);
    gx[19] = 0.0f;
    gy[19] = 0.0f;
    gz[19] = YlmC::c4e * (140.0f * z2 - 60.0f) * z;
    gx[20] = YlmC::c4d * z * (7.0f * z2 - 3.0f);
    gy[20] = 0.0f;
    gz[20] = YlmC::c4d * x * (21.0f * z2 - 3.0f);
    gx[21] = YlmC::c4f * 2.0f * x * (7.0f * z2 - 1.0f);
    gy[21] = -YlmC::c4f * 2.0f * y * (7.0f * z2 - 1.0f);
    gz[21] = YlmC::c4f * 14.0f * z * (x2 - y2);
    gx[22] = YlmC::c4b * 3.0f * z * (x2 - y2);
    gy[22] = -YlmC::c4b * 6.0f * x * y * z;
    gz[22] = YlmC::c4b * x * (x2 - 3.0f * y2);
    gx[23] = YlmC::c4g * 4.0f * x * (x2 - 3.0f * y2);
    gy[23] = YlmC::c4g * 4.0f * y * (y2 - 3.0f * x2);
    gz[23] = 0.0f;
}

// Calls f(lm, Y_lm, dP/dx, dP/dy, dP/dz) for lm = 0..23 with the same polynomials as
// ylm_val / ylm_grad, one (l, m) at a time, so that callers keep only running sums live.
template <class F>
__device__ __forceinline__ void ylm_each(float x, float y, float z, F &&f) {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    const float xy = x * y, yz = y * z, xz = x * z;
    const float a5 = 5.0f * z2 - 1.0f, b7 = 7.0f * z2 - 1.0f, c7 = 7.0f * z2 - 3.0f;
    const float d2 = x2 - y2;
    f(0, YlmC::c1 * y, 0.0f, YlmC::c1, 0.0f);
    f(1, YlmC::c1 * z, 0.0f, 0.0f, YlmC::c1);
    f(2, YlmC::c1 * x, YlmC::c1, 0.0f, 0.0f);
    f(3, YlmC::c2a * xy, YlmC::c2a * y, YlmC::c2a * x, 0.0f);
    f(4, YlmC::c2a * yz, 0.0f, YlmC::c2a * z, YlmC::c2a * y);
    f(5, YlmC::c2b * (3.0f * z2 - 1.0f), 0.0f, 0.0f, YlmC::c2b * 6.0f * z);
    f(6, YlmC::c2a * xz, YlmC::c2a * z, 0.0f, YlmC::c2a * x);
    f(7, YlmC::c2c * d2, YlmC::c2c * 2.0f * x, -YlmC::c2c * 2.0f * y, 0.0f);
    f(8, YlmC::c3a * y * (3.0f * x2 - y2), YlmC::c3a * 6.0f * xy, YlmC::c3a * 3.0f * d2, 0.0f);
    f(9, YlmC::c3b * xy * z, YlmC::c3b * yz, YlmC::c3b * xz, YlmC::c3b * xy);
    f(10, YlmC::c3c * y * a5, 0.0f, YlmC::c3c * a5, YlmC::c3c * 10.0f * yz);
    f(11, YlmC::c3d * z * (5.0f * z2 - 3.0f), 0.0f, 0.0f, YlmC::c3d * (15.0f * z2 - 3.0f));
    f(12, YlmC::c3c * x * a5, YlmC::c3c * a5, 0.0f, YlmC::c3c * 10.0f * xz);
    f(13, YlmC::c3e * z * d2, YlmC::c3e * 2.0f * xz, -YlmC::c3e * 2.0f * yz, YlmC::c3e * d2);
    f(14, YlmC::c3a * x * (x2 - 3.0f * y2), YlmC::c3a * 3.0f * d2, -YlmC::c3a * 6.0f * xy, 0.0f);
    f(15, YlmC::c4a * xy * d2, YlmC::c4a * y * (3.0f * x2 - y2), YlmC::c4a * x * (x2 - 3.0f * y2), 0.0f);
    f(16, YlmC::c4b * yz * (3.0f * x2 - y2), YlmC::c4b * 6.0f * xy * z, YlmC::c4b * 3.0f * z * d2,
      YlmC::c4b * y * (3.0f * x2 - y2));
    f(17, YlmC::c4c * xy * b7, YlmC::c4c * y * b7, YlmC::c4c * x * b7, YlmC::c4c * 14.0f * xy * z);
    f(18, YlmC::c4d * yz * c7, 0.0f, YlmC::c4d * z * c7, YlmC::c4d * y * (21.0f * z2 - 3.0f));
    f(19, YlmC::c4e * ((35.0f * z2 - 30.0f) * z2 + 3.0f), 0.0f, 0.0f, YlmC::c4e * (140.0f * z2 - 60.0f) * z);
    f(20, YlmC::c4d * xz * c7, YlmC::c4d * z * c7, 0.0f, YlmC::c4d * x * (21.0f * z2 - 3.0f));
    f(21, YlmC::c4f * d2 * b7, YlmC::c4f * 2.0f * x * b7, -YlmC::c4f * 2.0f * y * b7, YlmC::c4f * 14.0f * z * d2);
    f(22, YlmC::c4b * xz * (x2 - 3.0f * y2), YlmC::c4b * 3.0f * z * d2, -YlmC::c4b * 6.0f * xy * z,
      YlmC::c4b * x * (x2 - 3.0f * y2));
    f(23, YlmC::c4g * (x2 * (x2 - 3.0f * y2) - y2 * (3.0f * x2 - y2)), YlmC::c4g * 4.0f * x * (x2 - 3.0f * y2),
      YlmC::c4g * 4.0f * y * (y2 - 3.0f * x2), 0.0f);
}

__device__ __forceinline__ int l_of_lm(int lm) { return lm < 3 ? 1 : lm < 8 ? 2 : lm < 15 ? 3 : 4; }

// 4-body scale in the real l = 2 basis.  The descriptor is the (2 2 2) Wigner-3j
// contraction of the complex l = 2 moments; in terms of the traceless symmetric
// matrix Mt = sum_m a_m E_m built from the real moments a_m (E_m the orthonormal
// basis that maps Y_2m to r^r^T - I/3) it equals KAPPA_REAL tr(Mt^3) with
// KAPPA_REAL = -(9/2) sqrt(2/35) (5/(4 pi))^{3/2} (8 pi/15)^{3/2} = -(9/2) sqrt(2/35) (2/3)^{3/2}.
constexpr float KAPPA_REAL = -0.58554004376911990f;

// Mt from the real l = 2 moments a[0..4] (m = -2..2):
//   [[a2/s2 - a0/s6, a-2/s2, a1/s2], [a-2/s2, -a2/s2 - a0/s6, a-1/s2], [a1/s2, a-1/s2, 2 a0/s6]]
// stored symmetric as (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void l2_matrix(const float *a, float *M) {
    const float is2 = 0.70710678118654752f, is6 = 0.40824829046386302f;
    M[0] = a[4] * is2 - a[2] * is6;
    M[1] = -a[4] * is2 - a[2] * is6;
    M[2] = 2.0f * a[2] * is6;
    M[3] = a[0] * is2;
    M[4] = a[3] * is2;
    M[5] = a[1] * is2;
}

// Product of two symmetric matrices, symmetrised: S = (A B + B A) / 2 in (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void sym_prod(const float *A, const float *B, float *S) {
    // full entries
    const float a00 = A[0], a11 = A[1], a22 = A[2], a01 = A[3], a02 = A[4], a12 = A[5];
    const float b00 = B[0], b11 = B[1], b22 = B[2], b01 = B[3], b02 = B[4], b12 = B[5];
    const float p00 = a00 * b00 + a01 * b01 + a02 * b02;
    const float p11 = a01 * b01 + a11 * b11 + a12 * b12;
    const float p22 = a02 * b02 + a12 * b12 + a22 * b22;
    const float p01 = a00 * b01 + a01 * b11 + a02 * b12;
    const float p10 = a01 * b00 + a11 * b01 + a12 * b02;
    const float p02 = a00 * b02 + a01 * b12 + a02 * b22;
    const float p20 = a02 * b00 + a12 * b01 + a22 * b02;
    const float p12 = a01 * b02 + a11 * b12 + a12 * b22;
    const float p21 = a02 * b01 + a12 * b11 + a22 * b12;
    S[0] = p00;
    S[1] = p11;
    S[2] = p22;
    S[3] = 0.5f * (p01 + p10);
    S[4] = 0.5f * (p02 + p20);
    S[5] = 0.5f * (p12 + p21);
}

// Projections <X, E_m> of a symmetric matrix onto the real l = 2 basis, m = -2..2.
__device__ __forceinline__ void l2_project(const float *X, float *p) {
    const float s2 = 1.41421356237309505f, is2 = 0.70710678118654752f, is6 = 0.40824829046386302f;
    p[0] = s2 * X[3];
    p[1] = s2 * X[5];
    p[2] = (2.0f * X[2] - X[0] - X[1]) * is6;
    p[3] = s2 * X[4];
    p[4] = (X[0] - X[1]) * is2;
}

__device__ __forceinline__ float sym_trace_prod(const float *A, const float *B) {  // tr(A B)
    return A[0] * B[0] + A[1] * B[1] + A[2] * B[2] + 2.0f * (A[3] * B[3] + A[4] * B[4] + A[5] * B[5]);
}

// Ziegler-Biersack-Littmark screened Coulomb term of one pair (Sec. "Training": ZBL
// support as in NEP; the universal screening function of the ZBL treatise):
//   V = kzz phi(r/a) / r,  phi(x) = 0.1818 e^{-3.2x} + 0.5099 e^{-0.9423x} + 0.2802 e^{-0.4029x}
//       + 0.02817 e^{-0.2016x},  kzz = e^2/(4 pi eps0) Z_i Z_j,  a = 0.8854 a_0/(Z_i^0.23 + Z_j^0.23),
// times the switch f_s = 1 below r1, (1 + cos(pi (r - r1)/(r2 - r1)))/2 up to r2.  Called for
// r < r2 only; e = f_s V, de = d(f_s V)/dr.  Hardware exponential and sine/cosine: a few
// ulp, far inside the FP32 path's tolerance.
__device__ __forceinline__ void zbl_term(float r, float kzz, float inv_a, float r1, float r2, float &e, float &de) {
    const float x = r * inv_a;
    const float t0 = 0.1818f * __expf(-3.2f * x), t1 = 0.5099f * __expf(-0.9423f * x);
    const float t2 = 0.2802f * __expf(-0.4029f * x), t3 = 0.02817f * __expf(-0.2016f * x);
    const float phi = (t0 + t1) + (t2 + t3);
    const float dphi = -inv_a * ((3.2f * t0 + 0.9423f * t1) + (0.4029f * t2 + 0.2016f * t3));
    const float rinv = 1.0f / r;
    const float v = kzz * phi * rinv;
    const float dv = kzz * (dphi - phi * rinv) * rinv;
    float f = 1.0f, fp = 0.0f;
    if (r >= r1) {
        const float w = r2 - r1;
        float sn, cs;
        __sincosf(PI_F * (r - r1) / w, &sn, &cs);  // argument in [0, pi]
        f = 0.5f * (1.0f + cs);
        fp = -0.5f * sn * PI_F / w;
    }
    e = f * v;
    de = f * dv + fp * v;
}

// 1/|d| for a pair displacement (hardware reciprocal square root, <= 2 ulp).
__device__ __forceinline__ float inv_norm(float r2) { return rsqrtf(r2); }

// Requests the cache lines of [p, p + bytes) into L2 ahead of use.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes, int lane, int nlanes) {
    const char *c = (const char *)((uintptr_t)p & ~(uintptr_t)127);
    const char *e = (const char *)p + bytes;
    for (const char *q = c + 128 * lane; q < e; q += 128 * nlanes) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

// Record k of a pair list of length n through the read-only path, or a zero record past
// the end: pair loops load the record of their next iteration one iteration ahead.
__device__ __forceinline__ float4 pair_or_zero(const float4 *pr, int k, int n) {
    return k < n ? __ldg(pr + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ int pair_j(float4 p) { return __float_as_int(p.w) >> 4; }
__device__ __forceinline__ int pair_t(float4 p) { return __float_as_int(p.w) & 15; }

// Same inclusion predicate as the neighbour build: float (dx*dx + dy*dy) + dz*dz < rc*rc
// with no fused multiply-add, on the stored float displacement.
__device__ __forceinline__ bool within(float4 p, float rc2) {
    const float xx = __fmul_rn(p.x, p.x), yy = __fmul_rn(p.y, p.y), zz = __fmul_rn(p.z, p.z);
    return __fadd_rn(__fadd_rn(xx, yy), zz) < rc2;
}

}  // namespace nep
