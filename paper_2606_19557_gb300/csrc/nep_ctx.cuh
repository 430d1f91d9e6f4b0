// Host-side context of the NEP library: device buffers, cached batch, schedule and graphs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nep_gb300.h"
#include "nep_internal.cuh"

namespace nep {

// Grow-only device buffer.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    // 0 on success, 1 on allocation failure
    int ensure_bytes(size_t b) {
        if (b == 0) b = 16;
        if (b <= bytes) return 0;
        release();
        if (cudaMalloc(&ptr, b) != cudaSuccess) {
            ptr = nullptr;
            cudaGetLastError();
            return 1;
        }
        bytes = b;
        return 0;
    }
    template <class T>
    int ensure(int64_t n) { return ensure_bytes(sizeof(T) * (size_t)(n > 0 ? n : 1)); }
    template <class T>
    T *as() const { return (T *)ptr; }
};

// Launch shape of one per-atom kernel and its static schedule.
struct Sched {
    int var = 0;         // kernel variant (KernelSet): lanes per atom and register budget
    int wpb = 4;         // warps per block
    int blocks = 0;      // grid size
    int W = 0;           // total warps
    DevBuf warp_begin;   // [W+1]
    DevBuf type_wlo, type_whi;  // [T] first / last warp holding each species (adjoint slots)
};

constexpr int NET_CHUNK = 128;  // work positions per network chunk of the whole batch
constexpr int NVAR = 6;
constexpr int NVAR_TUNE = 4;  // variants the whole-batch autotune tries (32 lanes per atom pays only
                              // for small mini-batch groups, whose own tuning includes it)

enum KernelId {
    KID_EXPAND = 0, KID_DESC, KID_NETFWD, KID_PAIR, KID_TERMS, KID_ADJ, KID_NETREV, KID_ADJCG, KID_ANN, KID_GRAD,
    KID_COUNT
};

struct Ctx;

// Per-bucket kernel entry points (compile-time shapes).
struct KernelSet {
    int NR, KR, NA, KA;
    // variants v = 0..5: lanes per atom sw[v] (8, 16 or 32), register budget v & 1
    // (0: blocks of <= 128 threads, 4 per SM, 128 registers; 1: 5 per SM, 96 registers)
    const void *fwd_fn[NVAR];   // forward pair-gradient stage
    const void *desc_fn[NVAR];  // forward descriptor stage
    const void *net_fwd_fn[2];  // network forward pass (one block per chunk): 64- and 16-row tiles
    size_t (*net_fwd_smem)(int NN);  // of the 64-row tiles (the larger)
    const void *adj_fn[NVAR];   // adjoint coefficient-gradient stage (the larger footprint)
    const void *jvp_fn[NVAR];   // adjoint JVP stage
    const void *net_rev_fn[2];  // network reverse pass (one block per chunk): 64- and 16-row tiles
    size_t (*net_rev_smem)(int NN);  // of the 64-row tiles (the larger)
    int max_wpb[NVAR];                   // largest warps per block each variant allows
    int sw[NVAR];
    size_t (*fwd_smem[NVAR])(int T, int NN);  // bytes per warp
    size_t (*adj_smem[NVAR])(int T, int NN);
    // forward stages (0 descriptors, 1 network, 2 pair gradients; -1 all)
    void (*launch_fwd[NVAR])(const AtomArgs &, int blocks, int wpb, int stage, cudaStream_t, bool pdl);
    // adjoint stages (0 JVP, 1 network reverse, 2 coefficient gradient; -1 all)
    void (*launch_adj[NVAR])(const AtomArgs &, int blocks, int wpb, int stage, cudaStream_t, bool pdl);
};

const KernelSet *select_kernels(int nR, int kR, int nA, int kA);

struct Ctx {
    nep_config cfg{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sm = 0;
    std::string err;

    // sizes (compact = user layout, padded = kernel layout)
    int T = 1, NN = 1, ND = 1, NDP = 1;
    int nR = 1, kR = 1, nA = 1, kA = 1;
    int64_t P = 0;
    ParOff po{};
    const KernelSet *ks = nullptr;
    std::vector<int> desc_map;  // compact descriptor index -> padded index
    DevBuf d_desc_map, d_desc_inv;

    // parameters
    DevBuf theta, qscale, par;
    bool have_params = false;

    // batch
    int64_t n_struct = 0, n_atoms = 0, n_pairs = 0, n_pairs_ang = 0;
    bool have_batch = false;
    DevBuf atom_off, pos, type, cell, struct_of;
    std::vector<int64_t> h_atom_off, h_nbr_off;
    std::vector<int> h_type, h_nang;
    bool h_lists_ok = false;  // h_nbr_off / h_nang hold the current lists (fetch_host_lists)

    // neighbour build
    DevBuf geom, nbins, bin_off, bin_cnt, bin_start, bin_cur, atom_bin, atom_wrap, bin_atoms, cnt, n_ang, nbr_off;
    DevBuf keys_tmp, keys, pair, rev, shift, scan_tmp, d_total, d_err;
    DevBuf pos4, nbr_scratch, d_flag;  // float4 positions, per-atom key scratch, overflow flag
    DevBuf bin_pos, bin_wrap;          // atoms in bin order: (x, y, z, bits(j)) and wrap offsets
    int64_t nbin_total = 0;            // bins of the current cells
    bool geom_ok = false;              // geom / nbins / bin_off / struct_of hold the current cells
    // candidate lists for position updates with the cells kept (pairs within r_c + skin of
    // the reference positions cand_ref); grid for the wider cutoff in cgeom / cnbins / cbin_off
    float skin = 0.5f;                 // Angstrom; 0: every position update scans
    bool cand_ok = false, cgeom_ok = false;
    int64_t cand_M = 0, cnbin_total = 0;
    DevBuf cgeom, cnbins, cbin_off, cand_off, cand_key, cand_rev, cand_pidx, cand_flag, cand_ref, cand_rec;

    // schedule
    DevBuf work;                 // [Na] atom per work position (species-sorted)
    std::vector<int> h_work, type_begin;  // type_begin [T+1] work positions
    DevBuf rec, rec2;  // work records of `work` (int4 atom / first pair / pair counts, int2 species / structure)
    Sched fwd, adj;
    DevBuf sched_cost, sched_pre;  // [Na + 1] work cost per position and its exclusive prefix
    // network-gradient contraction chunks
    int n_chunks = 0;
    DevBuf chunk_begin, chunk_type, type_clo, type_chi;

    // per-step buffers
    DevBuf E_atom, F_own, W_atom, G, st_qt, st_h, st_A;
    DevBuf st_D, st_S, st_b, st_ab;   // adjoint stage outputs (JVP of A, radial species sums, b, abar)
    DevBuf st_E;                      // network energy per work position
    DevBuf fbar, ebar, wbar, zt, ut, om, dqt, cpart, annpart;
    DevBuf F_int, E_int, W_int;       // internal outputs for nep_loss_grad
    DevBuf loss_part, gb1, n_sv, loss3_int, grad_int;
    DevBuf gpart;                     // [8][P] FP64 segment sums of the gradient reduction
    // arrival counters of the last-block reductions (zero between launches; the last block
    // of a launch resets its counter): [0] loss terms, [1] optimiser, [2..] gradient columns
    DevBuf counters;
    DevBuf tgt_E, tgt_F, tgt_W, tgt_hw;  // nep_set_targets copies
    bool have_targets = false, tgt_has_hw = false;
    std::vector<int64_t> tgt_nsv_pre;    // [ns + 1] prefix count of the structures with virial targets
    // programmatic dependent launch between the step's kernels (NEP_PDL=1): measured no
    // faster on the step graphs, whose kernels are long against the launch gaps
    bool use_pdl = false;
    bool pdl() const { return use_pdl && !timing; }
    DevBuf hostbuf_theta;             // device copy target of nep_loss_grad_host

    // ZBL short-range term (nep_set_zbl): per species pair e^2/(4 pi eps0) Z_i Z_j and 1/a_ij
    DevBuf zbl_tab;
    float zbl_r1 = 0.0f, zbl_r2 = 0.0f;  // zbl_r2 = 0: off

    // loss normalisers (0 = this batch's own N_s, N_a, N_s^V); set for one shard of a batch
    double ov_Ns = 0.0, ov_Na = 0.0, ov_NsV = 0.0;
    double norm_Ns() const { return ov_Ns > 0.0 ? ov_Ns : (double)n_struct; }
    double norm_Na() const { return ov_Na > 0.0 ? ov_Na : (double)n_atoms; }

    // optimiser (AMSGrad + plateau schedule); state slots OPT_*
    bool have_opt = false;
    nep_optim_config ocfg{};
    DevBuf opt_m, opt_v, opt_vmax, opt_st;

    // mini-batch mode: groups of consecutive structures, each with its own schedule
    struct MiniBatch {
        int64_t s0, s1, a0, a1;  // structure and atom ranges (work positions = [a0, a1))
        int Wf, Wa;              // warps of the forward / adjoint launch (multiples of wpb)
        int64_t wf_off, wa_off;  // offsets of the warp_begin slices in mb_wbf / mb_wba
        int64_t ck_off;          // offset of the chunk list in mb_chunks (n_ck + 1 entries)
        int n_ck;
        int ch;                  // work positions per chunk (the last of a species may be shorter)
    };
    int mb_B = 0;
    int mb_var[2] = {-1, -1};  // forward / adjoint variants of the groups (-1: the batch's own)
    int mb_used[4] = {0, 0, 0, 0};  // variants and warps per block the schedules use
    int mb_key[6] = {-1, -1, -1, -1, -1, -1};  // launch shapes the schedules were built for
    std::vector<MiniBatch> mb;
    DevBuf mb_work, mb_wbf, mb_wba, mb_wlo, mb_whi, mb_chunks, mb_clo, mb_chi;
    DevBuf mb_rec, mb_rec2;  // work records of mb_work
    std::vector<cudaGraphExec_t> mb_graphs;  // per group: training step, captured on first use
    std::vector<uint64_t> mb_gkey;           // loss weights the graphs were captured with

    int schedule = NEP_SCHED_PERSISTENT;
    // plain form (per-structure launches)
    bool plain_ready = false;
    std::vector<int64_t> p_cofs;
    DevBuf p_work, p_ident, p_wlo, p_whi, p_clo, p_chi, p_chunks, p_acc, p_part;
    DevBuf p_rec, p_rec2;  // work records of p_work
    bool state_valid = false;

    // graphs
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<const void *> key;
        bool timing = false;
    };
    Graph g_loss, g_eval, g_train;
    bool timing = false;
    cudaEvent_t ev[KID_COUNT + 1] = {};
    bool ev_made = false;
    bool last_timed = false;

    int fail(int code, const char *msg) {
        err = msg;
        return code;
    }
    int fail_cuda(cudaError_t e, const char *where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return NEP_ECUDA;
    }
    ~Ctx();
};

#define CK(x)                                                      \
    do {                                                           \
        cudaError_t e_ = (x);                                      \
        if (e_ != cudaSuccess) return c->fail_cuda(e_, #x);        \
    } while (0)

// Launch check that names the kernel in the error message.
#define CK_LAUNCH(name)                                                   \
    do {                                                                  \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return c->fail_cuda(e_, "launch of " name); \
    } while (0)

int scan_exclusive(Ctx *c, const int64_t *in, int64_t n, int64_t *out, int64_t *total_dev);
// same_cells: the cells are those of the previous successful build (geometry kept);
// host_lists: copy the per-atom counts and offsets to h_nang / h_nbr_off.
int build_neighbors(Ctx *c, bool same_cells = false, bool host_lists = true);
// candidate lists (nep_neighbor.cu): build at the current positions, and the exact lists
// from them; moved_too_far: some atom moved half the skin or more (nothing valid written)
int build_candidates(Ctx *c);
int filter_candidates(Ctx *c, bool host_lists, bool &moved_too_far);
int fetch_host_lists(Ctx *c);

// step pieces (nep_loss.cu)
// Work records of a work order (after the neighbour lists and the order are final): per
// position the atom, its first pair and pair counts, its species and structure.
int build_work_rec(Ctx *c, const int *work, DevBuf &rec, DevBuf &rec2);
int launch_expand(Ctx *c);
int launch_forward(Ctx *c, float *q_raw, int stage = -1);
// explicit schedules (mini-batch mode)
int launch_forward_sched(Ctx *c, const int *work, const DevBuf &rec, const DevBuf &rec2, const int *warp_begin,
                         int blocks, int var, int wpb, const int *chunks, int n_chunks, int chunk_rows);
int launch_adjoint_sched(Ctx *c, const int *work, const DevBuf &rec, const DevBuf &rec2, const int *warp_begin,
                         int blocks, int var, int wpb, const int *chunks, int n_chunks, int chunk_rows);
int launch_ann_grad_chunks(Ctx *c, const int *chunks, int n_chunks);
// opt: apply the optimiser step to each parameter as its gradient completes (training)
int launch_grad_final_sched(Ctx *c, float *grad, const int *clo, const int *chi, const int *wlo, const int *whi,
                            const int *warp_begin, bool opt, const double *loss3, double lE, double lF, double lV);
// One launch of the force gather (atoms [a0, a1)), the per-structure sums (structures
// [s0, s1)) and, with loss3, the loss reduction by the launch's last block.
struct TermsCall {
    int64_t a0 = 0, a1 = 0, s0 = 0, s1 = 0;
    float *F_out = nullptr;
    double *E_out = nullptr, *W_out = nullptr;
    bool loss = false;  // loss terms and cotangents against the references below
    const float *F_ref = nullptr;
    const double *E_ref = nullptr, *W_ref = nullptr;
    const uint8_t *has_W = nullptr;
    double lE = 0.0, lF = 0.0, lV = 0.0;
    double nsv = 0.0;         // N_s^V: > 0 given; 0 counted here from has_W over [s0, s1); < 0 the
                              // count an earlier launch_count_hasw left on the device
    double *loss3 = nullptr;  // null: partials only (reduced later by launch_loss_final)
    double *fpart = nullptr;  // force partials, one per gather block (null: the context's loss_part)
    double *spart = nullptr;  // structure partials, 3 per structure (null: after the force partials)
    int gather_blocks = 0;    // 0: the default
    bool pdl = true;          // programmatic dependent launch (when the context allows it)
};
int launch_terms(Ctx *c, const TermsCall &t);
// N_s^V of structures [s0, s1) for the loss, known on the host: has_W absent or the
// targets' copy; 0 if it must be counted on the device.  A range without virial targets
// gives 1 (any positive value: no virial term enters then).
double host_nsv(Ctx *c, const uint8_t *has_W, int64_t s0, int64_t s1);
int launch_loss_final(Ctx *c, double *loss3, const double *fpart, int nf, const double *spart, int nsb, double nsv);
int launch_count_hasw(Ctx *c, const uint8_t *has_W, int64_t s0, int64_t s1);
int run_plain_loss(Ctx *c, const double *Er, const float *Fr, const double *Wr, const uint8_t *hw, double lE,
                   double lF, double lV, double *loss3, float *grad);
int launch_cotangents(Ctx *c, const double *dE, const float *dF, const double *dW);
int launch_adjoint(Ctx *c, int stage = -1);
int launch_ann_grad(Ctx *c);
int launch_grad_final(Ctx *c, float *grad, bool opt = false, const double *loss3 = nullptr, double lE = 0.0,
                      double lF = 0.0, double lV = 0.0);
int launch_range(Ctx *c, const float *q, float *qmin, float *qmax);

// optimiser (nep_optim.cu); device state slots
enum { OPT_T, OPT_B1T, OPT_B2T, OPT_LR, OPT_BEST, OPT_BAD, OPT_ACC, OPT_NACC, OPT_LAST, OPT_NRED, OPT_NST };

// Refresh of the padded parameter copies (par) from one compact parameter theta[k]: the
// inverse of the expansion, so an update keeps par in step with theta without a launch.
struct ParScatter {
    ParOff po;
    int T, NN, ND, NDP, nR, kR, nA, kA, NRP, KRP, NAP, KAP;
    const int *map;  // [ND] compact -> padded descriptor index
    float *par;
};

__device__ inline void scatter_param(const ParScatter &s, int64_t k, float v) {
    const int T = s.T, NN = s.NN, ND = s.ND;
    const int64_t cb0 = (int64_t)T * NN * ND, cw1 = cb0 + (int64_t)T * NN, cb1 = cw1 + (int64_t)T * NN;
    const int64_t ccR = cb1 + 1, ccA = ccR + (int64_t)T * T * s.nR * s.kR;
    if (k < cb0) {
        const int64_t tm = k / ND;  // t * NN + mu
        const int vp = s.map[(int)(k - tm * ND)];
        const int t = (int)(tm / NN), mu = (int)(tm - (int64_t)t * NN);
        s.par[s.po.w0 + tm * s.NDP + vp] = v;
        s.par[s.po.w0t + ((int64_t)t * s.NDP + vp) * NN + mu] = v;
    } else if (k < cw1) {
        s.par[s.po.b0 + (k - cb0)] = v;
    } else if (k < cb1) {
        s.par[s.po.w1 + (k - cw1)] = v;
    } else if (k == cb1) {
        s.par[s.po.b1] = v;
    } else if (k < ccA) {
        const int64_t r = k - ccR;
        const int kk = (int)(r % s.kR), n = (int)((r / s.kR) % s.nR);
        const int64_t ab = r / ((int64_t)s.kR * s.nR);
        s.par[s.po.cR + (ab * s.NRP + n) * s.KRP + kk] = v;
        s.par[s.po.cRp + (ab * s.NRP + n) * round4(s.KRP) + kk] = v;
    } else {
        const int64_t r = k - ccA;
        const int kk = (int)(r % s.kA), n = (int)((r / s.kA) % s.nA);
        const int64_t ab = r / ((int64_t)s.kA * s.nA);
        s.par[s.po.cA + (ab * s.NAP + n) * s.KAP + kk] = v;
        s.par[s.po.cAp + (ab * s.NAP + n) * round4(s.KAP) + kk] = v;
    }
}

// One AMSGrad step (the update rule of the optimiser file) inside another kernel.
struct OptArgs {
    float *theta;
    double *m, *v, *vmax, *st;
    double b1, b2, eps;
    const double *loss3;  // the step's loss terms for the epoch mean (or loss1, or neither)
    double lE, lF, lV;
    const double *loss1;
    ParScatter ps;
};

// State of this step as every element sees it (the tick is written once, afterwards).
struct OptStep {
    double bc1, bc2, lr;
};
__device__ inline OptStep opt_step_state(const OptArgs &o) {
    OptStep s;
    s.bc1 = 1.0 - o.st[OPT_B1T] * o.b1;
    s.bc2 = 1.0 - o.st[OPT_B2T] * o.b2;
    s.lr = o.st[OPT_LR];
    return s;
}
__device__ inline void amsgrad_elem(const OptArgs &o, const OptStep &s, int64_t i, double gi) {
    const double mi = __dadd_rn(__dmul_rn(o.b1, o.m[i]), __dmul_rn(1.0 - o.b1, gi));
    const double vi = __dadd_rn(__dmul_rn(o.b2, o.v[i]), __dmul_rn(__dmul_rn(1.0 - o.b2, gi), gi));
    o.m[i] = mi;
    o.v[i] = vi;
    const double vh = vi / s.bc2;
    const double vm = o.vmax[i] > vh ? o.vmax[i] : vh;
    o.vmax[i] = vm;
    const double step = __dmul_rn(s.lr, mi / s.bc1) / __dadd_rn(sqrt(vm), o.eps);
    const float th = (float)__dadd_rn((double)o.theta[i], -step);
    o.theta[i] = th;
    scatter_param(o.ps, i, th);
}
// Step counter, beta powers and the epoch loss sum: one thread, after every element's update.
__device__ inline void opt_tick(const OptArgs &o) {
    o.st[OPT_T] += 1.0;
    o.st[OPT_B1T] *= o.b1;
    o.st[OPT_B2T] *= o.b2;
    if (o.loss3) {
        o.st[OPT_ACC] += o.lE * o.loss3[0] + o.lF * o.loss3[1] + o.lV * o.loss3[2];
        o.st[OPT_NACC] += 1.0;
    } else if (o.loss1) {
        o.st[OPT_ACC] += o.loss1[0];
        o.st[OPT_NACC] += 1.0;
    }
}

// Last-block arrival: every thread of the block calls it, wrote = this thread stored data
// that the last block will read; true in the block that arrived last (it reads the other
// blocks' data through L2, __ldcg).
__device__ inline bool last_block_arrival(unsigned *counter, unsigned nblocks, bool wrote) {
    __shared__ unsigned s_last;
    if (wrote) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const bool last = atomicAdd(counter, 1u) == nblocks - 1u;
        if (last) *counter = 0u;  // every other block has arrived: ready for the next launch
        s_last = last ? 1u : 0u;
    }
    __syncthreads();
    return s_last != 0u;
}

// Unevaluated pair sums in FP32 (hi + lo): the FP32 pipes run 64x the FP64 rate on this
// part, and a compensated sum of FP32 terms keeps the error of an FP64 sum (Knuth's
// TwoSum: the rounding error of each addition is carried in lo).  Fixed order, so
// deterministic like the FP64 reductions they replace.
__device__ __forceinline__ void f2_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}
__device__ __forceinline__ void f2_merge(float &hi, float &lo, float h2, float l2) {
    f2_add(hi, lo, h2);
    lo += l2;
}

OptArgs opt_args(Ctx *c, const double *loss3, double lE, double lF, double lV, const double *loss1);
ParScatter par_scatter(Ctx *c);
int launch_opt_reset(Ctx *c);
int launch_opt_set_lr(Ctx *c, double lr);
int launch_opt_step(Ctx *c, const float *grad, const double *loss3, double lE, double lF, double lV,
                    const double *loss1);
int launch_opt_epoch(Ctx *c);

// mini-batch mode (nep_minibatch.cu)
int build_minibatches(Ctx *c, int batch_size);
int minibatch_shape_check(Ctx *c);  // rebuilds the schedules if the launch shape changed
int minibatch_tune(Ctx *c);         // picks the kernel variants of the group steps by timing
void drop_minibatch_graphs(Ctx *c);
void drop_graphs(Ctx *c);  // every cached graph (whole-batch and mini-batch)
// opt: training step (optimiser update fused into the gradient reduction)
int run_minibatch_loss(Ctx *c, int64_t m, double lE, double lF, double lV, double *loss3, float *grad,
                       bool opt = false);
int prepare_loss_kernels(Ctx *c);

}  // namespace nep
