/*
 * nep_gb300.h -- C ABI of the GB300 (sm_103a) NEP loss + parameter-gradient hot path.
 *
 * The model is the neuroevolution potential as stated in the TorchNEP paper
 * (arXiv 2606.19557): per-atom energies (Eq. 1) from a per-species one-hidden-
 * layer tanh network (Eq. "ann") on normalised descriptors (Eq. "norm") built
 * from Chebyshev radial functions and angular moments (Methods, "NEP
 * descriptors"), trained on the energy/force/virial loss (Eq. "loss") with
 * analytic parameter gradients (Sec. "Training efficiency ...": closed-form
 * expressions from the descriptor-coordinate Jacobian instead of a second-order
 * autograd pass).
 *
 * Conventions for every entry point
 *   - Return value: NEP_OK (0) or a negative NEP_E* code.  No exception or
 *     signal crosses the ABI.  nep_last_error() gives a one-line reason.  A call
 *     that fails argument validation changes nothing in the context.
 *   - Pointers named *_dev are DEVICE pointers on the context's GPU, owned by the
 *     caller; they must stay valid until the work queued by the call has
 *     finished on the context's stream.  Pointers named *_host are host pointers
 *     (pinned or pageable), owned by the caller.  The context owns only its
 *     internal workspaces.
 *   - Execution: calls queue work on the stream given to nep_create() and
 *     return without waiting, except where a description says "synchronizes".
 *   - Units: Angstrom, eV, eV/Angstrom; virials in eV.
 *   - Limits: 1 <= n_types <= 16; 0 <= n_max <= 11; 0 <= basis_size <= 11;
 *     0 <= l_max <= 4 (4-body needs l_max >= 2, 5-body l_max >= 1);
 *     1 <= n_neuron <= 128; 0 < rc_A <= rc_R; fewer than 2^27 atoms and 2^31
 *     neighbour pairs per context; every structure holds at least one atom.
 *
 * Parameter vector theta (float32, P entries; nep_num_params gives P):
 *   [ w0 : T x N_neu x N_des | b0 : T x N_neu | w1 : T x N_neu | b1 : 1 |
 *     cR : T x T x N_R x K_R | cA : T x T x N_A x K_A ]
 * with N_R = n_max_R + 1, K_R = basis_R + 1 (same for A), coefficients c
 * indexed [t_i][t_j][n][k] for the ordered species pair of the centre atom i and
 * neighbour j (Methods, g_n = sum_k c^{t_i t_j}_{nk} f_k).  This reproduces the
 * parameter counts of Table 2 (70,401 / 97,537 / 124,673).
 * Descriptor order (N_des = N_R + N_A (l_max + has_4b + has_5b)):
 *   [ q_n (N_R) | q_nl for l = 1..l_max, n fastest | q4_n | q5_n ].
 */
#ifndef NEP_GB300_H
#define NEP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEP_OK 0
#define NEP_EINVAL (-1)   /* invalid argument, unsupported size, or bad geometry           */
#define NEP_ENOMEM (-2)   /* device or host allocation failed                              */
#define NEP_ECUDA (-3)    /* a CUDA runtime call failed (message in nep_last_error)        */
#define NEP_ESTATE (-4)   /* call out of order (e.g. nep_eval before nep_set_structures)   */
#define NEP_EINTERNAL (-5)/* an internal consistency check on the device failed            */

#define NEP_PREC_FP32 0   /* FP32 pair/network arithmetic, FP64 structure and batch sums    */

#define NEP_SCHED_PERSISTENT 0 /* one persistent launch per kernel over all structures, graph */
#define NEP_SCHED_PLAIN 1      /* one launch sequence per structure, no graph (baseline form) */

typedef struct nep_ctx nep_ctx;

/* Model hyper-parameters: the model keys of the NEP input file (Table 1: type,
 * cutoff, n_max, basis_size, l_max, neuron).  has_4b / has_5b are the second and
 * third l_max entries ("4 2 1") as flags. */
typedef struct {
    int n_types;
    float rc_R, rc_A;
    int n_max_R, n_max_A;
    int basis_R, basis_A;
    int l_max, has_4b, has_5b;
    int n_neuron;
    int precision; /* NEP_PREC_FP32 */
    int device;    /* CUDA device ordinal */
} nep_config;

/* Creates a context on cfg->device that queues its work on `cuda_stream` (a
 * cudaStream_t).  With NULL the context creates a non-blocking stream of its own
 * (destroyed with it); the legacy default stream cannot be used because the loss
 * pass is captured into a CUDA graph.  *out receives the handle.
 * Errors: NEP_EINVAL (sizes outside the limits above), NEP_ECUDA, NEP_ENOMEM. */
int nep_create(const nep_config *cfg, void *cuda_stream, nep_ctx **out);

/* Frees every workspace of the context (synchronizes its stream).  NULL is a no-op. */
void nep_destroy(nep_ctx *ctx);

/* P, the length of theta (layout above).  Errors: NEP_EINVAL (NULL arguments). */
int nep_num_params(const nep_ctx *ctx, int64_t *P);

/* N_des, the descriptor length.  Errors: NEP_EINVAL. */
int nep_num_descriptors(const nep_ctx *ctx, int *n_des);

/* Copies theta_dev [P] (float32) and the normalisation factors q_scale_dev
 * [N_des] (float32, s_nu = 1/(q_nu^max - q_nu^min), Eq. "norm") into the context.
 * The copy is queued on the stream; the caller's buffers may be reused once it
 * has run.  Errors: NEP_EINVAL (NULL), NEP_ECUDA. */
int nep_set_params(nep_ctx *ctx, const float *theta_dev, const float *q_scale_dev);

/* Caches a batch of periodic structures and builds their neighbour lists (cell
 * lists -> CSR) once, as the paper keeps neighbour lists and displacement vectors
 * resident on the GPU (Sec. "Training efficiency ...").
 *   atom_off_dev [n_struct+1] int64: atoms of structure s are atom_off[s]..atom_off[s+1]-1
 *   pos_dev      [N_a*3] float32 Cartesian positions (any image; need not be wrapped)
 *   type_dev     [N_a] int32 species in [0, n_types)
 *   cell_dev     [n_struct*9] float32 row-major 3x3 cells, rows = lattice vectors
 * A pair (i, j, S) is a neighbour iff d = r_j + S.h - r_i, formed in FP64 and
 * rounded once to float, has float d.d < rc_R^2 (radial) / < rc_A^2 (angular);
 * j = i is included for S != 0.  n_struct = 0 is valid (empty batch).
 * Synchronizes.  Errors: NEP_EINVAL (counts, species, non-finite positions,
 * singular cell, more than 127 periodic images per direction), NEP_ENOMEM,
 * NEP_ECUDA. */
int nep_set_structures(nep_ctx *ctx, int64_t n_struct, const int64_t *atom_off_dev, const float *pos_dev,
                       const int32_t *type_dev, const float *cell_dev);

/* New positions (and optionally cells) for the cached batch: same structures, atom
 * counts and species.  pos_dev [N_a*3] f32 (device); cell_dev [n_struct*9] f32 (device)
 * or NULL to keep the cells (their bin grids are then reused).  Rebuilds the neighbour
 * lists on the device (as an MD-style evaluation needs every step) and
 * re-balances the per-atom kernel schedules for the new neighbour counts with the same
 * launch shapes, so every later result equals that of a fresh context on the new
 * geometry, bit for bit.  Without mini-batches the schedules are built on the device;
 * with them (nep_minibatch_setup) the group schedules are rebuilt on the host.
 * With the cells kept and a nonzero skin (nep_set_skin) the lists come from candidate
 * lists: every pair within r_c^R + skin of the positions at the last candidate scan.
 * While no atom has moved half the skin from those positions, the lists are the
 * candidates that pass the pair predicate at the new positions (a filter, no scan); the
 * filter keeps the scan's order, so the lists are the scan's, bit for bit.  Otherwise
 * the candidates are rebuilt first.  The candidate lists take about 33 bytes per
 * candidate pair.  Synchronizes with the list build; the schedule kernels are queued on
 * the context's stream after it.  Errors: NEP_ESTATE (no batch), NEP_EINVAL (bad
 * geometry: the batch is then unusable, and later calls return NEP_ESTATE, until
 * nep_set_structures), NEP_ENOMEM, NEP_ECUDA. */
int nep_update_positions(nep_ctx *ctx, const float *pos_dev, const float *cell_dev);

/* Skin (Angstrom, in [0, 10]; default 0.5) of the candidate lists of nep_update_positions
 * with the cells kept; 0 scans on every update.  The paper keeps neighbour lists on the
 * GPU (Sec. "Training efficiency"); the skin is this implementation's way to refresh them
 * between MD-style steps.  Errors: NEP_EINVAL. */
int nep_set_skin(nep_ctx *ctx, float skin);

/* Radial and angular neighbour-pair counts of the cached batch. */
int nep_num_pairs(const nep_ctx *ctx, int64_t *n_radial, int64_t *n_angular);

/* Exports the cached neighbour list (for checks): nbr_off_dev [N_a+1] int64 CSR
 * offsets, j_dev [M] int32 neighbour atom, shift_dev [M*3] int32 image S,
 * ang_dev [M] uint8 (1 if within rc_A).  Within an atom, angular neighbours come
 * first, each group sorted by (species, j, S).  Errors: NEP_ESTATE, NEP_EINVAL. */
int nep_get_neighbors(nep_ctx *ctx, int64_t *nbr_off_dev, int32_t *j_dev, int32_t *shift_dev, uint8_t *ang_dev);

/* Energies, forces and virials at the current parameters (Eq. 1, Eq. "ann").
 *   E_dev [n_struct] float64, F_dev [N_a*3] float32 (F = -dE/dr),
 *   W_dev [n_struct*9] float64 with W = -dE/d(eps) for r -> (I + eps) r applied
 *   to positions and cell, i.e. W_ab = -sum_pairs (dE_i/dd_ij)_a (d_ij)_b.
 * Also stores the per-atom state nep_backward needs.
 * Errors: NEP_ESTATE (no structures or parameters), NEP_EINVAL, NEP_ECUDA. */
int nep_eval(nep_ctx *ctx, double *E_dev, float *F_dev, double *W_dev);

/* Raw descriptors q [N_a*N_des] float32 (before the scale of Eq. "norm"). */
int nep_descriptors(nep_ctx *ctx, float *q_dev);

/* Per-component minimum and maximum of q over the cached batch, [N_des] each
 * (helper for the normalisation factors of Eq. "norm"). */
int nep_descriptor_range(nep_ctx *ctx, float *qmin_dev, float *qmax_dev);

/* Same result as nep_descriptor_range, for callers that cannot allocate device memory
 * during the call: code running while a stream is being captured into a CUDA graph
 * (where cudaMalloc/cudaFree are not allowed), hosts whose own memory manager owns
 * every device allocation, or latency-critical loops that must not enter the driver's
 * allocator.  The paper has no counterpart; it is a library-interface addition.
 * The call allocates and frees nothing: the raw descriptors go to a fixed scratch array
 * of 8,388,608 floats (32 MiB) that lives in the library for the whole process on every
 * GPU that loads it.  Batches with N_a x (padded descriptor length) above that size are
 * rejected with NEP_EINVAL (the message gives the limit).  The first call on a device
 * looks up the array's device address; make that first call before any stream capture.
 * All calls share the one array, so calls whose GPU work overlaps (other streams,
 * other contexts on the same GPU) race; calls queued on one stream are safe.  Queued on
 * the context's stream, without waiting.  Errors: NEP_ESTATE, NEP_EINVAL, NEP_ECUDA. */
int nep_descriptor_range_noalloc(nep_ctx *ctx, float *qmin_dev, float *qmax_dev);

/* One full loss + parameter-gradient pass (Eq. "loss"):
 *   DE = 1/N_s sum_s ((E_s - E_ref_s)/N_a^s)^2
 *   DF = 1/(3 N_a) sum_i |F_i - F_ref_i|^2
 *   DV = 1/(9 N_s^V) sum_{s: has_W} |(W_s - W_ref_s)/N_a^s|^2   (0 if N_s^V = 0)
 *   L  = lamE DE + lamF DF + lamV DV
 *   E_ref_dev [n_struct] f64, F_ref_dev [N_a*3] f32, W_ref_dev [n_struct*9] f64,
 *   has_W_dev [n_struct] uint8 or NULL (= all structures have virials).
 * Writes loss3_dev [3] float64 = (DE, DF, DV) and grad_dev [P] float32 = dL/dtheta.
 * With NEP_SCHED_PERSISTENT the whole pass is one CUDA-graph launch.
 * Errors: NEP_ESTATE, NEP_EINVAL, NEP_ECUDA. */
int nep_loss_grad(nep_ctx *ctx, const double *E_ref_dev, const float *F_ref_dev, const double *W_ref_dev,
                  const uint8_t *has_W_dev, double lamE, double lamF, double lamV, double *loss3_dev,
                  float *grad_dev);

/* Normalisers of Eq. "loss" for a batch that is one shard of a larger one: N_s, N_a
 * and N_s^V of the whole batch (0 = use this context's own counts, the default).  With
 * them, the loss terms and gradients of the shards add up to those of the whole batch,
 * so one sum over shards (e.g. an all-reduce across GPUs) gives the full-batch pass.
 * Errors: NEP_EINVAL (negative or non-finite). */
int nep_set_loss_normalizers(nep_ctx *ctx, double N_s, double N_a, double N_s_V);

/* Ziegler-Biersack-Littmark short-range repulsion added to the energies, forces and
 * virials (Sec. "Training": TorchNEP supports ZBL as NEP does, citing the ZBL
 * treatise; the paper prints no formula).  Pair term, from the treatise's universal
 * screening function:
 *   V(r) = (e^2/(4 pi eps0)) Z_i Z_j phi(r/a) / r,  a = 0.8854 a_0 / (Z_i^0.23 + Z_j^0.23),
 *   phi(x) = 0.1818 e^{-3.2x} + 0.5099 e^{-0.9423x} + 0.2802 e^{-0.4029x} + 0.02817 e^{-0.2016x},
 * times the switch f_s = 1 for r < r1, (1 + cos(pi (r - r1)/(r2 - r1)))/2 for r1 <= r < r2,
 * 0 beyond; each ordered neighbour pair (i, j) adds f_s V / 2 to E_i.  The term has no
 * trainable parameter: it shifts E, F, W and the loss residuals, not the form of the
 * gradient.  Z_host [n_types] (host, atomic numbers in (0, 200)), 0 <= r1 < r2 <= rc_R;
 * r2 = 0 switches the term off (the default).  Takes effect from the next call.
 * Errors: NEP_EINVAL (values out of range), NEP_ENOMEM, NEP_ECUDA. */
int nep_set_zbl(nep_ctx *ctx, float r1, float r2, const float *Z_host);

/* Vector-Jacobian product for autograd (the analytic route of Sec. "Training
 * efficiency": the parameter gradient through the descriptor-coordinate Jacobian,
 * without a second-order autograd pass): grad_dev [P] = d/dtheta of
 *   sum_s dE_s E_s + sum_i dF_i . F_i + sum_s dW_s : W_s
 * with cotangents dE_dev [n_struct] f64, dF_dev [N_a*3] f32, dW_dev [n_struct*9] f64.
 * Uses the per-atom state of the latest nep_eval, which must have run with the
 * same parameters and structures.  Errors: NEP_ESTATE, NEP_EINVAL, NEP_ECUDA. */
int nep_backward(nep_ctx *ctx, const double *dE_dev, const float *dF_dev, const double *dW_dev, float *grad_dev);

/* Copies loss references into context-owned device buffers so that the host
 * entry point below needs none per call (same layouts as nep_loss_grad). */
int nep_set_targets(nep_ctx *ctx, const double *E_ref_dev, const float *F_ref_dev, const double *W_ref_dev,
                    const uint8_t *has_W_dev);

/* Host-buffer step: copies theta_host [P] to the device, runs nep_loss_grad on
 * the references of nep_set_targets, and copies loss3_host [3] and grad_host [P]
 * back.  Synchronizes.  The copies use the context's stream.
 * Errors: NEP_ESTATE (no targets), NEP_EINVAL, NEP_ECUDA. */
int nep_loss_grad_host(nep_ctx *ctx, const float *theta_host, double lamE, double lamF, double lamV,
                       double *loss3_host, float *grad_host);

/* ---------------------------------------------------------------- training loop
 * Optimiser of Sec. "Training": Adam with the AMSGrad variant that keeps the maximum
 * of the BIAS-CORRECTED second moment,
 *   m_t = b1 m + (1-b1) g,  v_t = b2 v + (1-b2) g^2,  m^ = m_t/(1-b1^t),  v^ = v_t/(1-b2^t),
 *   v^max = max(v^max, v^),  theta -= eta m^ / (sqrt(v^max) + eps),
 * applied to the context's own parameter copy (set by nep_set_params), and the
 * epoch-level plateau schedule eta <- max(factor eta, lr_min) after `patience`
 * consecutive epochs whose mean loss L_e fails L_e < best (1 - threshold).
 * Parameters stay FP32; moments and update arithmetic are FP64 on the device.  All
 * state lives on the device, so steps need no host round trip. */
typedef struct {
    double lr;        /* eta at the start (and after nep_optim_set_lr), > 0 */
    double beta1;     /* [0, 1), paper: 0.9 */
    double beta2;     /* [0, 1), paper: 0.999 */
    double eps;       /* >= 0, paper: 1e-8 */
    double factor;    /* plateau reduction gamma, (0, 1) */
    int patience;     /* p >= 1 consecutive epochs without improvement */
    double lr_min;    /* floor of eta, >= 0 */
    double threshold; /* relative improvement threshold tau, [0, 1) */
} nep_optim_config;

/* Zeroes the moments, sets t = 0 and eta = cfg->lr, forgets the best loss.
 * Errors: NEP_EINVAL (a value out of range), NEP_ENOMEM, NEP_ECUDA. */
int nep_optim_init(nep_ctx *ctx, const nep_optim_config *cfg);

/* One optimiser step on the context's parameters with gradient grad_dev [P] f32
 * (device).  loss_dev (device, 1 double, or NULL) is added to the epoch's loss sum.
 * Asynchronous on the context's stream.  Errors: NEP_ESTATE (no nep_optim_init). */
int nep_optim_step(nep_ctx *ctx, const float *grad_dev, const double *loss_dev);

/* One training step on the whole cached batch: nep_loss_grad at the current
 * parameters against the references of nep_set_targets (weights lamE, lamF, lamV),
 * then the optimiser step; the step's loss L = lamE DE + lamF DF + lamV DV joins the
 * epoch sum.  One CUDA graph.  loss3_dev (device [3] or NULL) receives DE, DF, DV
 * at the parameters BEFORE the update.  Errors: NEP_ESTATE, NEP_EINVAL, NEP_ECUDA. */
int nep_train_step(nep_ctx *ctx, double lamE, double lamF, double lamV, double *loss3_dev);

/* Epoch boundary: mean loss of the steps since the previous boundary, improvement
 * test and, after `patience` bad epochs, the rate reduction (all on the device). */
int nep_optim_epoch_end(nep_ctx *ctx);

/* Start of a stage of the two-stage protocol: eta = lr and the plateau schedule
 * restarts (best loss forgotten); moments and t are kept.  Errors: NEP_EINVAL. */
int nep_optim_set_lr(nep_ctx *ctx, double lr);

/* Optimiser state, copied to the host (synchronizes): out_host[6] = t, eta, best
 * epoch loss, bad epochs, latest epoch loss (NaN before the first), reductions. */
int nep_optim_state(nep_ctx *ctx, double *out_host);

/* Copies the context's current parameters into theta_dev [P] f32 (device). */
int nep_get_params(nep_ctx *ctx, float *theta_dev);

/* ---------------------------------------------------------------- mini-batch mode
 * Sec. "Training": every optimisation step uses a mini-batch of structures while the
 * geometry (neighbour lists, pair records) of the whole cached batch is built once.
 * nep_minibatch_setup splits the cached batch into groups of batch_size CONSECUTIVE
 * structures (the last group may be smaller; shuffle the structures before
 * nep_set_structures to randomise the composition) and builds each group's kernel
 * schedule on the host, once.  *n_batches (may be NULL) receives the group count.
 * Invalidated by nep_set_structures.  Errors: NEP_ESTATE, NEP_EINVAL, NEP_ENOMEM. */
int nep_minibatch_setup(nep_ctx *ctx, int batch_size, int64_t *n_batches);

/* Loss and gradient of group m alone (normalisers N_s, N_a, N_s^V of the group)
 * against the references of nep_set_targets; outputs as nep_loss_grad (device). */
int nep_minibatch_loss_grad(nep_ctx *ctx, int64_t m, double lamE, double lamF, double lamV, double *loss3_dev,
                            float *grad_dev);

/* nep_minibatch_loss_grad of group m followed by the optimiser step; the group's
 * weighted loss joins the epoch sum.  loss3_dev: device [3] or NULL. */
int nep_minibatch_train_step(nep_ctx *ctx, int64_t m, double lamE, double lamF, double lamV, double *loss3_dev);

/* One epoch driven by the library: training steps on the groups order_host[0..n_steps)
 * in that order, then nep_optim_epoch_end.  Asynchronous (no host synchronisation).
 * Errors: NEP_EINVAL (an index out of range: nothing is launched). */
int nep_minibatch_epoch(nep_ctx *ctx, const int64_t *order_host, int64_t n_steps, double lamE, double lamF,
                        double lamV);

/* Selects NEP_SCHED_PERSISTENT (default) or NEP_SCHED_PLAIN. */
int nep_set_schedule(nep_ctx *ctx, int schedule);

/* Times launch shapes (warps per block, blocks per SM) of the two per-atom kernels
 * on the cached batch and keeps the fastest.  Synchronizes.  Results are
 * deterministic for a fixed shape; different shapes may differ in the last bits
 * of the gradient (another reduction tree). */
int nep_autotune(nep_ctx *ctx);

/* Current launch shape: warps per block and blocks of the forward and adjoint kernels. */
int nep_get_launch(const nep_ctx *ctx, int *fwd_warps, int *fwd_blocks, int *adj_warps, int *adj_blocks);

/* Kernel variant of the forward and adjoint kernels: lanes that share one atom (8, 16 or
 * 32) and the register budget per thread (128 or 96). */
int nep_get_variant(const nep_ctx *ctx, int *fwd_lanes, int *fwd_regs, int *adj_lanes, int *adj_regs);

/* Selects kernel variants v in [0, 6): lanes per atom 8 (v < 2), 16 (v < 4) or 32,
 * register budget 128 (v even) or 96 (v odd); the grid is reset to the occupancy limit.
 * nep_autotune tries v < 4; mini-batch setup also tries the 32-lane variants. */
int nep_set_variant(nep_ctx *ctx, int fwd_var, int adj_var);

/* Sets the launch shape explicitly (0 keeps a value); at most 4 warps per block. */
int nep_set_launch(nep_ctx *ctx, int fwd_warps, int fwd_blocks, int adj_warps, int adj_blocks);

/* Kernel timing: when on, the graph of nep_loss_grad records CUDA events around
 * each kernel; nep_kernel_times then returns, for the latest completed call, the
 * duration in ms of each kernel (names from nep_kernel_name).  n_io: in = capacity,
 * out = number written. */
int nep_set_timing(nep_ctx *ctx, int on);
int nep_kernel_times(nep_ctx *ctx, float *ms, int *n_io);
const char *nep_kernel_name(int k);

/* FP32 fused multiply-add throughput probe (measurement helper, no counterpart in the
 * paper): queues on cuda_stream (a cudaStream_t; NULL = legacy default stream) one
 * kernel of `blocks` blocks x 256 threads, each thread running 8 independent chains of
 * `iters` dependent FMAs.  *flops receives the kernel's floating-point operations
 * (2 per FMA); divided by the kernel's duration (CUDA events on the same stream) it is
 * the measured FP32 peak that the per-atom kernels' roofline fractions use.  Use a grid
 * of several blocks per SM (e.g. 8 x the SM count).  sink_dev: device float (never
 * written in practice; it keeps the arithmetic live).  Errors: NEP_EINVAL (blocks < 1,
 * iters not a positive multiple of 16, NULL pointers), NEP_ECUDA (launch failed). */
int nep_fp32_fma_probe(void *cuda_stream, int blocks, int64_t iters, float *sink_dev, double *flops);

/* Last error message of this context (or of the latest failed nep_create when ctx is NULL). */
const char *nep_last_error(const nep_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NEP_GB300_H */
