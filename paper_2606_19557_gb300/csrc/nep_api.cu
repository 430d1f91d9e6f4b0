// C ABI of the NEP library: context lifecycle, batch caching, static schedule,
// CUDA-graph capture of the loss + gradient pass, and the launch-shape autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "nep_ctx.cuh"

using namespace nep;

struct nep_ctx : public nep::Ctx {};

namespace nep {
int launch_compact_q(Ctx *c, const float *qp, float *q);

Ctx::~Ctx() {
    if (g_loss.exec) cudaGraphExecDestroy(g_loss.exec);
    if (g_eval.exec) cudaGraphExecDestroy(g_eval.exec);
    if (g_train.exec) cudaGraphExecDestroy(g_train.exec);
    drop_minibatch_graphs(this);
    if (ev_made)
        for (auto &e : ev) cudaEventDestroy(e);
}
}  // namespace nep

static thread_local std::string g_create_err;

static const char *kernel_names[KID_COUNT] = {"expand_params", "forward_desc", "net_forward", "forward_pair",
                                              "loss_terms",    "adjoint_jvp",  "net_reverse", "adjoint_cgrad",
                                              "net_grad",      "grad_reduce"};

// ----------------------------------------------------------------------------- helpers

static int check_cfg(const nep_config *c, std::string &why) {
    if (!c) return why = "null config", 0;
    if (c->n_types < 1 || c->n_types > TMAX) return why = "n_types must be in [1, 16]", 0;
    if (c->n_max_R < 0 || c->n_max_R > 11 || c->n_max_A < 0 || c->n_max_A > 11)
        return why = "n_max must be in [0, 11]", 0;
    if (c->basis_R < 0 || c->basis_R > 11 || c->basis_A < 0 || c->basis_A > 11)
        return why = "basis_size must be in [0, 11]", 0;
    if (c->l_max < 0 || c->l_max > 4) return why = "l_max must be in [0, 4]", 0;
    if (c->has_4b && c->l_max < 2) return why = "the 4-body term needs l_max >= 2", 0;
    if (c->has_5b && c->l_max < 1) return why = "the 5-body term needs l_max >= 1", 0;
    if (c->n_neuron < 1 || c->n_neuron > NNMAX) return why = "n_neuron must be in [1, 128]", 0;
    if (!(c->rc_R > 0.0f) || !(c->rc_A > 0.0f) || c->rc_A > c->rc_R || !(c->rc_R < 1e4f))
        return why = "cutoffs must satisfy 0 < rc_A <= rc_R", 0;
    if (c->precision != NEP_PREC_FP32) return why = "unsupported precision", 0;
    return 1;
}

// Static schedule of one per-atom kernel: contiguous ranges of the species-sorted work
// order with about equal cost per warp (cost ~ radial pairs + 6 x angular pairs + 8).
static int make_sched(Ctx *c, Sched &s, int wpb, int blocks, int var) {
    int rc = fetch_host_lists(c);
    if (rc) return rc;
    s.var = var;
    s.wpb = wpb;
    s.blocks = blocks;
    s.W = wpb * blocks;
    const int64_t na = c->n_atoms;
    std::vector<int> begin(s.W + 1, 0);
    if (na > 0) {
        std::vector<double> pre(na + 1, 0.0);
        for (int64_t q = 0; q < na; ++q) {
            const int i = c->h_work[q];
            const double nr = (double)(c->h_nbr_off[i + 1] - c->h_nbr_off[i]);
            pre[q + 1] = pre[q] + nr + 6.0 * c->h_nang[i] + 8.0;
        }
        const double tot = pre[na];
        int64_t q = 0;
        for (int w = 0; w <= s.W; ++w) {
            const double target = tot * (double)w / (double)s.W;
            while (q < na && pre[q] < target) ++q;
            begin[w] = (int)q;
        }
        begin[s.W] = (int)na;
        for (int w = 1; w <= s.W; ++w) begin[w] = std::max(begin[w], begin[w - 1]);
    }
    std::vector<int> wlo(c->T, 0), whi(c->T, -1);
    for (int t = 0; t < c->T; ++t) {
        const int p0 = c->type_begin[t], p1 = c->type_begin[t + 1];
        if (p1 <= p0) continue;
        // warp holding position p: the last w with begin[w] <= p < begin[w+1]
        auto owner = [&](int p) {
            int lo = 0, hi = s.W - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (begin[mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        wlo[t] = owner(p0);
        whi[t] = owner(p1 - 1);
    }
    if (s.warp_begin.ensure<int>(s.W + 1) || s.type_wlo.ensure<int>(c->T) || s.type_whi.ensure<int>(c->T))
        return c->fail(NEP_ENOMEM, "schedule buffers");
    CK(cudaMemcpy(s.warp_begin.ptr, begin.data(), sizeof(int) * (s.W + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.type_wlo.ptr, wlo.data(), sizeof(int) * c->T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.type_whi.ptr, whi.data(), sizeof(int) * c->T, cudaMemcpyHostToDevice));
    return NEP_OK;
}

// The same schedules built on the device from the current lists, without copying them to
// the host (used when only the positions changed).  The costs are integers, so their
// prefix is exact in int64 and in the host's doubles alike (below 2^53); the split targets
// take the same double operations, so the warp ranges equal those of make_sched.
namespace {
__global__ void k_sched_cost(int64_t na, const int *work, const int64_t *nbr_off, const int *n_ang, int64_t *cost) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= na) return;
    const int i = work[q];
    cost[q] = (nbr_off[i + 1] - nbr_off[i]) + 6 * (int64_t)n_ang[i] + 8;
}

// begin[w] = first work position q with pre[q] >= tot * w / W (na if none); begin[W] = na
__global__ void k_sched_split(int64_t na, const int64_t *pre, int W, int *begin) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w > W) return;
    if (w == W) {
        begin[W] = (int)na;
        return;
    }
    const double target = (double)pre[na] * (double)w / (double)W;
    int64_t lo = 0, hi = na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if ((double)pre[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    begin[w] = (int)lo;
}

struct TypeRanges {
    int begin[TMAX + 1];  // work positions of each species
};

// first / last warp holding each species: the last w with begin[w] <= p
__global__ void k_sched_types(int T, TypeRanges tr, const int *begin, int W, int *wlo, int *whi) {
    const int t = threadIdx.x;
    if (t >= T) return;
    const int p0 = tr.begin[t], p1 = tr.begin[t + 1];
    if (p1 <= p0) {
        wlo[t] = 0;
        whi[t] = -1;
        return;
    }
    auto owner = [&](int p) {
        int lo = 0, hi = W - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (begin[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    wlo[t] = owner(p0);
    whi[t] = owner(p1 - 1);
}
}  // namespace

static int make_scheds_device(Ctx *c) {
    const int64_t na = c->n_atoms;
    if (na == 0 || c->T > TMAX) {
        int rc = make_sched(c, c->fwd, c->fwd.wpb, c->fwd.blocks, c->fwd.var);
        return rc ? rc : make_sched(c, c->adj, c->adj.wpb, c->adj.blocks, c->adj.var);
    }
    if (c->sched_cost.ensure<int64_t>(na + 1) || c->sched_pre.ensure<int64_t>(na + 1))
        return c->fail(NEP_ENOMEM, "schedule workspace");
    const cudaStream_t st = c->stream;
    k_sched_cost<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(na, c->work.as<int>(), c->nbr_off.as<int64_t>(),
                                                              c->n_ang.as<int>(), c->sched_cost.as<int64_t>());
    CK(cudaGetLastError());
    int rc = scan_exclusive(c, c->sched_cost.as<int64_t>(), na, c->sched_pre.as<int64_t>(), c->d_total.as<int64_t>() + 2);
    if (rc) return rc;
    TypeRanges tr{};
    for (int t = 0; t <= c->T; ++t) tr.begin[t] = c->type_begin[t];
    for (Sched *s : {&c->fwd, &c->adj}) {
        s->W = s->wpb * s->blocks;
        if (s->warp_begin.ensure<int>(s->W + 1) || s->type_wlo.ensure<int>(c->T) || s->type_whi.ensure<int>(c->T))
            return c->fail(NEP_ENOMEM, "schedule buffers");
        k_sched_split<<<(unsigned)((s->W + 256) / 256), 256, 0, st>>>(na, c->sched_pre.as<int64_t>(), s->W,
                                                                       s->warp_begin.as<int>());
        k_sched_types<<<1, 32, 0, st>>>(c->T, tr, s->warp_begin.as<int>(), s->W, s->type_wlo.as<int>(),
                                        s->type_whi.as<int>());
        CK(cudaGetLastError());
    }
    return NEP_OK;
}

static int max_blocks_per_sm(Ctx *c, const void *fn, int wpb, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, wpb * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// The dynamic shared-memory limit is an attribute of the kernel (shared by every
// context in the process), so it is raised to the device maximum, never lowered.
static int set_smem_attr(Ctx *c) {
    int maxo = 0;
    CK(cudaDeviceGetAttribute(&maxo, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    if (c->ks->fwd_smem[2](c->T, c->NN) > (size_t)maxo || c->ks->adj_smem[2](c->T, c->NN) > (size_t)maxo)
        return c->fail(NEP_EINVAL, "model too large for shared memory");
    if (c->ks->net_rev_smem(c->NN) > (size_t)maxo || c->ks->net_fwd_smem(c->NN) > (size_t)maxo)
        return c->fail(NEP_EINVAL, "model too large for shared memory");
    for (int r = 0; r < 2; ++r) {
        CK(cudaFuncSetAttribute(c->ks->net_fwd_fn[r], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
        CK(cudaFuncSetAttribute(c->ks->net_rev_fn[r], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
    }
    for (int v = 0; v < NVAR; ++v) {
        CK(cudaFuncSetAttribute(c->ks->fwd_fn[v], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
        CK(cudaFuncSetAttribute(c->ks->desc_fn[v], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
        CK(cudaFuncSetAttribute(c->ks->adj_fn[v], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
        CK(cudaFuncSetAttribute(c->ks->jvp_fn[v], cudaFuncAttributeMaxDynamicSharedMemorySize, maxo));
    }
    return NEP_OK;
}

// Buffers whose size depends on the schedule (per-warp gradient partials).
static int alloc_sched_buffers(Ctx *c) {
    const int NC = c->ks->NR * c->ks->KR + c->ks->NA * c->ks->KA;
    if (c->cpart.ensure<float>((int64_t)(c->adj.W + c->T) * c->T * NC))
        return c->fail(NEP_ENOMEM, "gradient partials");
    return NEP_OK;
}

static int default_shapes(Ctx *c) {
    int rc = set_smem_attr(c);
    if (rc) return rc;
    if ((rc = prepare_loss_kernels(c))) return rc;
    // 16 lanes per atom, 128 registers; 4 warps per block, fewer when a large model's
    // shared-memory tail (it grows with the species count) does not fit
    const int v = 3;
    int wf = 0, wa = 0, bf = 0, ba = 0;
    for (int w = 4; w >= 1 && bf < 1; w /= 2)
        if ((bf = max_blocks_per_sm(c, c->ks->fwd_fn[v], w, c->ks->fwd_smem[v](c->T, c->NN) * w)) >= 1) wf = w;
    for (int w = 4; w >= 1 && ba < 1; w /= 2)
        if ((ba = max_blocks_per_sm(c, c->ks->adj_fn[v], w, c->ks->adj_smem[v](c->T, c->NN) * w)) >= 1) wa = w;
    if (bf < 1 || ba < 1) return c->fail(NEP_EINVAL, "kernel does not fit on the device (shared memory)");
    if ((rc = make_sched(c, c->fwd, wf, c->n_sm * bf, v))) return rc;
    if ((rc = make_sched(c, c->adj, wa, c->n_sm * ba, v))) return rc;
    return alloc_sched_buffers(c);
}

void nep::drop_graphs(Ctx *c) {
    for (Ctx::Graph *g : {&c->g_loss, &c->g_eval, &c->g_train}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        g->key.clear();
    }
    drop_minibatch_graphs(c);
}

static void mark(Ctx *c, int k) {
    if (c->timing) cudaEventRecordWithFlags(c->ev[k], c->stream, cudaEventRecordExternal);
}

// ----------------------------------------------------------------------------- step bodies

static int body_eval(Ctx *c, double *E, float *F, double *W) {
    int rc;
    if ((rc = launch_expand(c))) return rc;
    if ((rc = launch_forward(c, nullptr))) return rc;
    TermsCall t;
    t.a1 = c->n_atoms;
    t.s1 = c->n_struct;
    t.F_out = F;
    t.E_out = E;
    t.W_out = W;
    return launch_terms(c, t);
}

// opt: training step, the optimiser update fused into the gradient reduction
static int body_loss(Ctx *c, const double *Er, const float *Fr, const double *Wr, const uint8_t *hw, double lE,
                     double lF, double lV, double *loss3, float *grad, bool opt = false) {
    int rc;
    mark(c, 0);
    if ((rc = launch_expand(c))) return rc;
    mark(c, 1);
    if ((rc = launch_forward(c, nullptr, 0))) return rc;
    mark(c, 2);
    if ((rc = launch_forward(c, nullptr, 1))) return rc;
    mark(c, 3);
    if ((rc = launch_forward(c, nullptr, 2))) return rc;
    mark(c, 4);
    TermsCall t;
    t.a1 = c->n_atoms;
    t.s1 = c->n_struct;
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
    t.nsv = c->ov_NsV > 0.0 ? c->ov_NsV : host_nsv(c, hw, 0, c->n_struct);
    t.loss3 = loss3;
    if ((rc = launch_terms(c, t))) return rc;
    mark(c, 5);
    if ((rc = launch_adjoint(c, 0))) return rc;
    mark(c, 6);
    if ((rc = launch_adjoint(c, 1))) return rc;
    mark(c, 7);
    if ((rc = launch_adjoint(c, 2))) return rc;
    mark(c, 8);
    if ((rc = launch_ann_grad(c))) return rc;
    mark(c, 9);
    if ((rc = launch_grad_final(c, grad, opt, loss3, lE, lF, lV))) return rc;
    mark(c, 10);
    return NEP_OK;
}

// Runs `body` through a cached CUDA graph keyed by `key`.
template <class Fn>
static int run_graph(Ctx *c, Ctx::Graph &g, const std::vector<const void *> &key, Fn body) {
    if (!g.exec || g.key != key || g.timing != c->timing) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int rc = body();
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();  // clear the invalidated-capture status
            return rc;
        }
        if (e != cudaSuccess) return c->fail_cuda(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return c->fail_cuda(e, "cudaGraphInstantiate");
        }
        g.key = key;
        g.timing = c->timing;
    }
    CK(cudaGraphLaunch(g.exec, c->stream));
    return NEP_OK;
}

// ----------------------------------------------------------------------------- C ABI

extern "C" {

int nep_create(const nep_config *cfg, void *cuda_stream, nep_ctx **out) {
    std::string why;
    if (!out) return NEP_EINVAL;
    *out = nullptr;
    if (!check_cfg(cfg, why)) {
        g_create_err = why;
        return NEP_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        g_create_err = "no such CUDA device";
        return NEP_ECUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_err = "cudaSetDevice failed";
        return NEP_ECUDA;
    }
    nep_ctx *c = new (std::nothrow) nep_ctx();
    if (!c) return NEP_ENOMEM;
    c->cfg = *cfg;
    c->dev = cfg->device;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->dev);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_create_err = "cudaStreamCreate failed";
            delete c;
            return NEP_ECUDA;
        }
        c->own_stream = true;
    }
    c->T = cfg->n_types;
    c->NN = cfg->n_neuron;
    c->nR = cfg->n_max_R + 1;
    c->kR = cfg->basis_R + 1;
    c->nA = cfg->n_max_A + 1;
    c->kA = cfg->basis_A + 1;
    const int L = cfg->l_max, H4 = cfg->has_4b ? 1 : 0, H5 = cfg->has_5b ? 1 : 0;
    c->ND = c->nR + c->nA * (L + H4 + H5);
    c->ks = select_kernels(c->nR, c->kR, c->nA, c->kA);
    if (!c->ks) {
        g_create_err = "no kernel shape for these sizes";
        delete c;
        return NEP_EINVAL;
    }
    c->NDP = c->ks->NR + 6 * c->ks->NA;
    const int64_t T = c->T, NN = c->NN;
    c->P = T * NN * c->ND + 2 * T * NN + 1 + T * T * ((int64_t)c->nR * c->kR + (int64_t)c->nA * c->kA);
    c->po = par_offsets(c->T, c->NN, c->ks->NR, c->ks->KR, c->ks->NA, c->ks->KA);
    // compact -> padded descriptor map
    c->desc_map.clear();
    for (int n = 0; n < c->nR; ++n) c->desc_map.push_back(n);
    for (int l = 1; l <= L; ++l)
        for (int n = 0; n < c->nA; ++n) c->desc_map.push_back(c->ks->NR + (l - 1) * c->ks->NA + n);
    if (H4)
        for (int n = 0; n < c->nA; ++n) c->desc_map.push_back(c->ks->NR + 4 * c->ks->NA + n);
    if (H5)
        for (int n = 0; n < c->nA; ++n) c->desc_map.push_back(c->ks->NR + 5 * c->ks->NA + n);
    std::vector<int> inv(c->NDP, -1);
    for (int v = 0; v < c->ND; ++v) inv[c->desc_map[v]] = v;
    if (c->d_desc_map.ensure<int>(c->ND) || c->d_desc_inv.ensure<int>(c->NDP) || c->theta.ensure<float>(c->P) ||
        c->qscale.ensure<float>(c->ND) || c->par.ensure<float>(c->po.total) || c->d_err.ensure<int>(4) ||
        c->n_sv.ensure<int>(4) || c->gb1.ensure<double>(4) || c->loss3_int.ensure<double>(4) ||
        c->grad_int.ensure<float>(c->P) || c->hostbuf_theta.ensure<float>(c->P) ||
        c->gpart.ensure<double>(8 * c->P) || c->counters.ensure<unsigned>(3 + (c->P + 31) / 32)) {
        g_create_err = "device allocation failed";
        delete c;
        return NEP_ENOMEM;
    }
    if (cudaMemcpy(c->d_desc_map.ptr, c->desc_map.data(), sizeof(int) * c->ND, cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->d_desc_inv.ptr, inv.data(), sizeof(int) * c->NDP, cudaMemcpyHostToDevice) ||
        cudaMemset(c->counters.ptr, 0, c->counters.bytes)) {
        g_create_err = "cudaMemcpy failed";
        delete c;
        return NEP_ECUDA;
    }
    for (int k = 0; k <= KID_COUNT; ++k) cudaEventCreate(&c->ev[k]);
    c->ev_made = true;
    if (const char *e = getenv("NEP_PDL")) c->use_pdl = std::strcmp(e, "1") == 0;
    *out = c;
    return NEP_OK;
}

void nep_destroy(nep_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->stream);
    const bool own = c->own_stream;
    cudaStream_t st = c->stream;
    delete c;
    if (own) cudaStreamDestroy(st);
}

int nep_num_params(const nep_ctx *c, int64_t *P) {
    if (!c || !P) return NEP_EINVAL;
    *P = c->P;
    return NEP_OK;
}

int nep_num_descriptors(const nep_ctx *c, int *nd) {
    if (!c || !nd) return NEP_EINVAL;
    *nd = c->ND;
    return NEP_OK;
}

int nep_set_params(nep_ctx *c, const float *theta, const float *qscale) {
    if (!c) return NEP_EINVAL;
    if (!theta || !qscale) return c->fail(NEP_EINVAL, "null parameter pointer");
    CK(cudaSetDevice(c->dev));
    CK(cudaMemcpyAsync(c->theta.ptr, theta, sizeof(float) * c->P, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->qscale.ptr, qscale, sizeof(float) * c->ND, cudaMemcpyDeviceToDevice, c->stream));
    // the padded copies follow theta from here on (every optimiser update refreshes them)
    int rc = launch_expand(c);
    if (rc) return rc;
    c->have_params = true;
    c->state_valid = false;
    return NEP_OK;
}

int nep_set_structures(nep_ctx *c, int64_t ns, const int64_t *atom_off, const float *pos, const int32_t *type,
                       const float *cell) {
    if (!c) return NEP_EINVAL;
    if (ns < 0) return c->fail(NEP_EINVAL, "negative structure count");
    if (ns > 0 && (!atom_off || !pos || !type || !cell)) return c->fail(NEP_EINVAL, "null structure pointer");
    CK(cudaSetDevice(c->dev));
    CK(cudaDeviceSynchronize());
    std::vector<int64_t> off(ns + 1, 0);
    if (ns > 0) CK(cudaMemcpy(off.data(), atom_off, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost));
    if (off[0] != 0) return c->fail(NEP_EINVAL, "atom_off[0] must be 0");
    for (int64_t s = 0; s < ns; ++s)
        if (off[s + 1] - off[s] < 1) return c->fail(NEP_EINVAL, "every structure needs at least one atom");
    const int64_t na = off[ns];
    if (na >= ((int64_t)1 << 27)) return c->fail(NEP_EINVAL, "too many atoms (limit 2^27)");
    drop_graphs(c);
    c->have_batch = false;
    c->state_valid = false;
    c->have_targets = false;
    c->plain_ready = false;
    c->mb.clear();
    c->mb_B = 0;
    c->n_struct = ns;
    c->n_atoms = na;
    if (c->atom_off.ensure<int64_t>(ns + 1) || c->pos.ensure<float>(na * 3) || c->type.ensure<int>(na) ||
        c->cell.ensure<float>(ns * 9) || c->struct_of.ensure<int>(na))
        return c->fail(NEP_ENOMEM, "batch buffers");
    CK(cudaMemcpy(c->atom_off.ptr, off.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
    if (na > 0) {
        CK(cudaMemcpy(c->pos.ptr, pos, sizeof(float) * 3 * na, cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(c->type.ptr, type, sizeof(int) * na, cudaMemcpyDeviceToDevice));
    }
    if (ns > 0) CK(cudaMemcpy(c->cell.ptr, cell, sizeof(float) * 9 * ns, cudaMemcpyDeviceToDevice));
    c->h_atom_off = off;
    int rc = build_neighbors(c);
    if (rc) return rc;
    // species-sorted work order
    c->h_type.assign(na, 0);
    if (na > 0) CK(cudaMemcpy(c->h_type.data(), c->type.ptr, sizeof(int) * na, cudaMemcpyDeviceToHost));
    c->h_work.resize(na);
    std::iota(c->h_work.begin(), c->h_work.end(), 0);
    std::stable_sort(c->h_work.begin(), c->h_work.end(), [&](int x, int y) { return c->h_type[x] < c->h_type[y]; });
    c->type_begin.assign(c->T + 1, 0);
    for (int64_t i = 0; i < na; ++i) c->type_begin[c->h_type[i] + 1]++;
    for (int t = 0; t < c->T; ++t) c->type_begin[t + 1] += c->type_begin[t];
    if (c->work.ensure<int>(na)) return c->fail(NEP_ENOMEM, "work order");
    if (na > 0) CK(cudaMemcpy(c->work.ptr, c->h_work.data(), sizeof(int) * na, cudaMemcpyHostToDevice));
    if ((rc = build_work_rec(c, c->work.as<int>(), c->rec, c->rec2))) return rc;
    // network-gradient chunks (single species each)
    {
        const int CH = NET_CHUNK;  // work positions per network chunk
        std::vector<int> cb, clo(c->T), chi(c->T);
        for (int t = 0; t < c->T; ++t) {
            clo[t] = (int)cb.size();
            for (int p = c->type_begin[t]; p < c->type_begin[t + 1]; p += CH) cb.push_back(p);
            chi[t] = (int)cb.size();
        }
        c->n_chunks = (int)cb.size();
        cb.push_back((int)na);
        if (c->chunk_begin.ensure<int>(cb.size()) || c->type_clo.ensure<int>(c->T) || c->type_chi.ensure<int>(c->T))
            return c->fail(NEP_ENOMEM, "chunk buffers");
        CK(cudaMemcpy(c->chunk_begin.ptr, cb.data(), sizeof(int) * cb.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->type_clo.ptr, clo.data(), sizeof(int) * c->T, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->type_chi.ptr, chi.data(), sizeof(int) * c->T, cudaMemcpyHostToDevice));
        if (c->annpart.ensure<float>((int64_t)(c->n_chunks + 1) * (c->NN * c->NDP + 2 * c->NN)))
            return c->fail(NEP_ENOMEM, "network partials");
    }
    // per-step buffers
    const int64_t M = c->n_pairs, NDP = c->NDP, NN = c->NN, NAL = (int64_t)c->ks->NA * L3;
    const int64_t nlp = (int64_t)c->n_sm * 4 + 3 * ns + 8;  // gather blocks + 3 per structure
    if (c->E_atom.ensure<float>(na) || c->F_own.ensure<float>(na * 3) || c->W_atom.ensure<float>(na * 9) ||
        c->G.ensure_bytes(sizeof(float4) * (size_t)(M + 1)) || c->st_qt.ensure<float>(na * NDP) ||
        c->st_h.ensure<float>(na * NN) || c->st_A.ensure<float>(na * NAL) || c->fbar.ensure<float4>(na) ||
        c->ebar.ensure<float>(ns) || c->wbar.ensure<float>(ns * 9) || c->zt.ensure<float>(na * NN) ||
        c->ut.ensure<float>(na * NN) || c->om.ensure<float>(na * NN) || c->dqt.ensure<float>(na * NDP) ||
        c->F_int.ensure<float>(na * 3) || c->E_int.ensure<double>(ns) || c->W_int.ensure<double>(ns * 9) ||
        c->loss_part.ensure<double>(nlp) || c->st_D.ensure<float>(na * NAL) ||
        c->st_S.ensure<float>(na * 2 * (int64_t)c->T * c->ks->KR) || c->st_b.ensure<float>(na * NDP) ||
        c->st_ab.ensure<float>(na * NDP) || c->st_E.ensure<float>(na))
        return c->fail(NEP_ENOMEM, "step buffers");
    if ((rc = default_shapes(c))) return rc;
    CK(cudaDeviceSynchronize());
    c->have_batch = true;
    return NEP_OK;
}

int nep_update_positions(nep_ctx *c, const float *pos, const float *cell) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures (call nep_set_structures)");
    if (c->n_atoms > 0 && !pos) return c->fail(NEP_EINVAL, "null positions");
    CK(cudaSetDevice(c->dev));
    const void *before[5] = {c->pair.ptr, c->rev.ptr, c->G.ptr, c->nbr_off.ptr, c->n_ang.ptr};
    if (c->n_atoms > 0)
        CK(cudaMemcpyAsync(c->pos.ptr, pos, sizeof(float) * 3 * c->n_atoms, cudaMemcpyDeviceToDevice, c->stream));
    if (cell && c->n_struct > 0)
        CK(cudaMemcpyAsync(c->cell.ptr, cell, sizeof(float) * 9 * c->n_struct, cudaMemcpyDeviceToDevice, c->stream));
    c->have_batch = false;  // until the lists are rebuilt
    c->state_valid = false;
    // the mini-batch schedules are built on the host from host copies of the lists
    const bool host_lists = c->mb_B > 0;
    int rc = NEP_OK;
    bool done = false;
    if (!cell && c->skin > 0.0f) {  // cells kept: filter the candidate lists (rescan when stale)
        bool far = true;
        if (c->cand_ok && (rc = filter_candidates(c, host_lists, far))) return rc;
        if (!far) {
            done = true;
        } else if ((rc = build_candidates(c)) == NEP_OK) {
            if ((rc = filter_candidates(c, host_lists, far))) return rc;
            if (far) return c->fail(NEP_EINTERNAL, "candidate filter after a fresh scan");
            done = true;
        } else if (rc != NEP_EINVAL) {
            return rc;
        }
        // NEP_EINVAL: cells too thin for the wider cutoff (or bad positions, which the scan
        // below reports): this context scans from now on
        if (!done) c->skin = 0.0f;
    }
    if (!done && (rc = build_neighbors(c, cell == nullptr, host_lists))) return rc;
    if (c->G.ensure_bytes(sizeof(float4) * (size_t)(c->n_pairs + 1))) return c->fail(NEP_ENOMEM, "pair gradients");
    if ((rc = build_work_rec(c, c->work.as<int>(), c->rec, c->rec2))) return rc;  // new pair ranges
    // re-balance the kernel schedules for the new neighbour counts (same sizes, same
    // buffers): the result is then the one a fresh context computes, bit for bit
    if (host_lists) {
        if ((rc = make_sched(c, c->fwd, c->fwd.wpb, c->fwd.blocks, c->fwd.var))) return rc;
        if ((rc = make_sched(c, c->adj, c->adj.wpb, c->adj.blocks, c->adj.var))) return rc;
        if ((rc = build_minibatches(c, c->mb_B))) return rc;
    } else if ((rc = make_scheds_device(c))) {
        return rc;
    }
    const void *after[5] = {c->pair.ptr, c->rev.ptr, c->G.ptr, c->nbr_off.ptr, c->n_ang.ptr};
    if (!std::equal(before, before + 5, after)) drop_graphs(c);  // graphs hold the old addresses
    c->plain_ready = false;
    c->have_batch = true;
    return NEP_OK;
}

int nep_set_skin(nep_ctx *c, float skin) {
    if (!c) return NEP_EINVAL;
    if (!(skin >= 0.0f) || !(skin <= 10.0f)) return c->fail(NEP_EINVAL, "skin must be in [0, 10] Angstrom");
    c->skin = skin;
    c->cand_ok = c->cgeom_ok = false;
    return NEP_OK;
}

int nep_num_pairs(const nep_ctx *c, int64_t *nr, int64_t *na) {
    if (!c || !nr || !na) return NEP_EINVAL;
    if (!c->have_batch) return NEP_ESTATE;
    *nr = c->n_pairs;
    *na = c->n_pairs_ang;
    return NEP_OK;
}

namespace {
__global__ void k_export(int64_t na, const int64_t *nbr_off, const int *n_ang, const float4 *pair,
                         const int32_t *shift, int32_t *j_out, int32_t *s_out, uint8_t *ang_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    for (int64_t p = nbr_off[i]; p < nbr_off[i + 1]; ++p) {
        const uint32_t sp = (uint32_t)shift[p];
        if (j_out) j_out[p] = pair_j(pair[p]);
        if (s_out) {
            s_out[3 * p] = (int)((sp >> 16) & 255) - 128;
            s_out[3 * p + 1] = (int)((sp >> 8) & 255) - 128;
            s_out[3 * p + 2] = (int)(sp & 255) - 128;
        }
        if (ang_out) ang_out[p] = (p - nbr_off[i] < n_ang[i]) ? 1 : 0;
    }
}
}  // namespace

int nep_get_neighbors(nep_ctx *c, int64_t *nbr_off, int32_t *j, int32_t *shift, uint8_t *ang) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures");
    CK(cudaSetDevice(c->dev));
    if (nbr_off)
        CK(cudaMemcpyAsync(nbr_off, c->nbr_off.ptr, sizeof(int64_t) * (c->n_atoms + 1), cudaMemcpyDeviceToDevice,
                           c->stream));
    if (c->n_atoms > 0)
        k_export<<<(unsigned)((c->n_atoms + 127) / 128), 128, 0, c->stream>>>(
            c->n_atoms, c->nbr_off.as<int64_t>(), c->n_ang.as<int>(), (const float4 *)c->pair.ptr,
            c->shift.as<int32_t>(), j, shift, ang);
    CK(cudaGetLastError());
    return NEP_OK;
}

static int ready(nep_ctx *c) {
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures (call nep_set_structures)");
    if (!c->have_params) return c->fail(NEP_ESTATE, "no parameters (call nep_set_params)");
    return NEP_OK;
}

int nep_eval(nep_ctx *c, double *E, float *F, double *W) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if ((c->n_struct > 0 && (!E || !W)) || (c->n_atoms > 0 && !F)) return c->fail(NEP_EINVAL, "null output");
    CK(cudaSetDevice(c->dev));
    if (c->schedule == NEP_SCHED_PLAIN) {
        rc = body_eval(c, E, F, W);
    } else {
        const bool t = c->timing;
        c->timing = false;
        rc = run_graph(c, c->g_eval, {E, F, W}, [&] { return body_eval(c, E, F, W); });
        c->timing = t;
    }
    if (rc) return rc;
    c->state_valid = true;
    return NEP_OK;
}

int nep_descriptors(nep_ctx *c, float *q) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (c->n_atoms > 0 && !q) return c->fail(NEP_EINVAL, "null output");
    CK(cudaSetDevice(c->dev));
    DevBuf qp;
    if (qp.ensure<float>(c->n_atoms * c->NDP)) return c->fail(NEP_ENOMEM, "descriptor buffer");
    if ((rc = launch_expand(c))) return rc;
    if ((rc = launch_forward(c, qp.as<float>(), 0))) return rc;
    if ((rc = launch_compact_q(c, qp.as<float>(), q))) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return NEP_OK;
}

int nep_descriptor_range(nep_ctx *c, float *qmin, float *qmax) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (!qmin || !qmax) return c->fail(NEP_EINVAL, "null output");
    CK(cudaSetDevice(c->dev));
    DevBuf qp;
    if (qp.ensure<float>(c->n_atoms * c->NDP)) return c->fail(NEP_ENOMEM, "descriptor buffer");
    if ((rc = launch_expand(c))) return rc;
    if ((rc = launch_forward(c, qp.as<float>(), 0))) return rc;
    if ((rc = launch_range(c, qp.as<float>(), qmin, qmax))) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return NEP_OK;
}

int nep_loss_grad(nep_ctx *c, const double *Er, const float *Fr, const double *Wr, const uint8_t *hw, double lE,
                  double lF, double lV, double *loss3, float *grad) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (!loss3 || !grad) return c->fail(NEP_EINVAL, "null output");
    if ((c->n_struct > 0 && (!Er || !Wr)) || (c->n_atoms > 0 && !Fr)) return c->fail(NEP_EINVAL, "null reference");
    if (!std::isfinite(lE) || !std::isfinite(lF) || !std::isfinite(lV)) return c->fail(NEP_EINVAL, "non-finite weight");
    CK(cudaSetDevice(c->dev));
    if (c->schedule == NEP_SCHED_PLAIN) {
        rc = run_plain_loss(c, Er, Fr, Wr, hw, lE, lF, lV, loss3, grad);
    } else {
        uint64_t lb[3];
        std::memcpy(&lb[0], &lE, 8);
        std::memcpy(&lb[1], &lF, 8);
        std::memcpy(&lb[2], &lV, 8);
        std::vector<const void *> key = {Er, Fr, Wr, hw, loss3, grad, (const void *)(uintptr_t)lb[0],
                                         (const void *)(uintptr_t)lb[1], (const void *)(uintptr_t)lb[2]};
        rc = run_graph(c, c->g_loss, key, [&] { return body_loss(c, Er, Fr, Wr, hw, lE, lF, lV, loss3, grad); });
        c->last_timed = c->timing;
    }
    if (rc) return rc;
    c->state_valid = true;
    return NEP_OK;
}

int nep_set_loss_normalizers(nep_ctx *c, double Ns, double Na, double NsV) {
    if (!c) return NEP_EINVAL;
    if (!(Ns >= 0.0) || !(Na >= 0.0) || !(NsV >= 0.0) || !std::isfinite(Ns + Na + NsV))
        return c->fail(NEP_EINVAL, "normalisers must be finite and >= 0");
    c->ov_Ns = Ns;
    c->ov_Na = Na;
    c->ov_NsV = NsV;
    drop_graphs(c);
    return NEP_OK;
}

int nep_set_zbl(nep_ctx *c, float r1, float r2, const float *Z) {
    if (!c) return NEP_EINVAL;
    if (r2 == 0.0f) {
        c->zbl_r1 = c->zbl_r2 = 0.0f;
        drop_graphs(c);
        c->state_valid = false;
        return NEP_OK;
    }
    if (!Z) return c->fail(NEP_EINVAL, "ZBL: atomic numbers missing");
    if (!(r1 >= 0.0f) || !(r2 > r1) || !(r2 <= c->cfg.rc_R))
        return c->fail(NEP_EINVAL, "ZBL: the switch radii must satisfy 0 <= r1 < r2 <= rc_R");
    for (int t = 0; t < c->T; ++t)
        if (!(Z[t] > 0.0f) || !(Z[t] < 200.0f)) return c->fail(NEP_EINVAL, "ZBL: atomic numbers must be in (0, 200)");
    const double ke = 14.399645, a0 = 0.52917721;  // e^2/(4 pi eps0) in eV A, Bohr radius in A
    std::vector<float> tab((size_t)c->T * c->T * 2);
    for (int i = 0; i < c->T; ++i)
        for (int j = 0; j < c->T; ++j) {
            const double zi = Z[i], zj = Z[j];
            tab[2 * (i * c->T + j)] = (float)(ke * zi * zj);
            tab[2 * (i * c->T + j) + 1] = (float)((std::pow(zi, 0.23) + std::pow(zj, 0.23)) / (0.8854 * a0));
        }
    CK(cudaSetDevice(c->dev));
    if (c->zbl_tab.ensure<float>((int64_t)tab.size())) return c->fail(NEP_ENOMEM, "ZBL table");
    CK(cudaMemcpy(c->zbl_tab.ptr, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
    c->zbl_r1 = r1;
    c->zbl_r2 = r2;
    drop_graphs(c);
    c->state_valid = false;
    return NEP_OK;
}

int nep_backward(nep_ctx *c, const double *dE, const float *dF, const double *dW, float *grad) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (!c->state_valid) return c->fail(NEP_ESTATE, "nep_backward needs a preceding nep_eval");
    if (!grad || (c->n_struct > 0 && (!dE || !dW)) || (c->n_atoms > 0 && !dF))
        return c->fail(NEP_EINVAL, "null pointer");
    CK(cudaSetDevice(c->dev));
    if ((rc = launch_cotangents(c, dE, dF, dW))) return rc;
    if ((rc = launch_adjoint(c))) return rc;
    if ((rc = launch_ann_grad(c))) return rc;
    if ((rc = launch_grad_final(c, grad))) return rc;
    return NEP_OK;
}

int nep_set_targets(nep_ctx *c, const double *Er, const float *Fr, const double *Wr, const uint8_t *hw) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures");
    const int64_t ns = c->n_struct, na = c->n_atoms;
    if ((ns > 0 && (!Er || !Wr)) || (na > 0 && !Fr)) return c->fail(NEP_EINVAL, "null reference");
    CK(cudaSetDevice(c->dev));
    if (c->tgt_E.ensure<double>(ns) || c->tgt_F.ensure<float>(na * 3) || c->tgt_W.ensure<double>(ns * 9) ||
        c->tgt_hw.ensure<uint8_t>(ns))
        return c->fail(NEP_ENOMEM, "target buffers");
    if (ns > 0) {
        CK(cudaMemcpyAsync(c->tgt_E.ptr, Er, sizeof(double) * ns, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->tgt_W.ptr, Wr, sizeof(double) * ns * 9, cudaMemcpyDeviceToDevice, c->stream));
        if (hw) CK(cudaMemcpyAsync(c->tgt_hw.ptr, hw, ns, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (na > 0) CK(cudaMemcpyAsync(c->tgt_F.ptr, Fr, sizeof(float) * na * 3, cudaMemcpyDeviceToDevice, c->stream));
    // N_s^V of any structure range from a host prefix count (loss normaliser of a group)
    c->tgt_nsv_pre.assign(ns + 1, 0);
    if (hw && ns > 0) {
        std::vector<uint8_t> h(ns);
        CK(cudaMemcpyAsync(h.data(), hw, ns, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int64_t s = 0; s < ns; ++s) c->tgt_nsv_pre[s + 1] = c->tgt_nsv_pre[s] + (h[s] ? 1 : 0);
    } else {
        for (int64_t s = 0; s < ns; ++s) c->tgt_nsv_pre[s + 1] = s + 1;
    }
    c->tgt_has_hw = hw != nullptr;
    c->have_targets = true;
    drop_graphs(c);  // the step graphs carry the normalisers of the previous targets
    return NEP_OK;
}

int nep_loss_grad_host(nep_ctx *c, const float *theta_host, double lE, double lF, double lV, double *loss3_host,
                       float *grad_host) {
    if (!c) return NEP_EINVAL;
    if (!c->have_targets) return c->fail(NEP_ESTATE, "no targets (call nep_set_targets)");
    if (!theta_host || !loss3_host || !grad_host) return c->fail(NEP_EINVAL, "null pointer");
    CK(cudaSetDevice(c->dev));
    CK(cudaMemcpyAsync(c->theta.ptr, theta_host, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream));
    if (!c->have_params) return c->fail(NEP_ESTATE, "no normalisation factors (call nep_set_params once)");
    int rc = nep_loss_grad(c, c->tgt_E.as<double>(), c->tgt_F.as<float>(), c->tgt_W.as<double>(),
                           c->tgt_has_hw ? c->tgt_hw.as<uint8_t>() : nullptr, lE, lF, lV, c->loss3_int.as<double>(),
                           c->grad_int.as<float>());
    if (rc) return rc;
    CK(cudaMemcpyAsync(loss3_host, c->loss3_int.ptr, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(grad_host, c->grad_int.ptr, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NEP_OK;
}

int nep_optim_init(nep_ctx *c, const nep_optim_config *o) {
    if (!c) return NEP_EINVAL;
    if (!o) return c->fail(NEP_EINVAL, "null optimiser configuration");
    const bool ok = std::isfinite(o->lr) && o->lr > 0.0 && o->beta1 >= 0.0 && o->beta1 < 1.0 && o->beta2 >= 0.0 &&
                    o->beta2 < 1.0 && std::isfinite(o->eps) && o->eps >= 0.0 && o->factor > 0.0 && o->factor < 1.0 &&
                    o->patience >= 1 && std::isfinite(o->lr_min) && o->lr_min >= 0.0 && o->threshold >= 0.0 &&
                    o->threshold < 1.0;
    if (!ok) return c->fail(NEP_EINVAL, "optimiser configuration out of range");
    CK(cudaSetDevice(c->dev));
    if (c->opt_m.ensure<double>(c->P) || c->opt_v.ensure<double>(c->P) || c->opt_vmax.ensure<double>(c->P) ||
        c->opt_st.ensure<double>(OPT_NST))
        return c->fail(NEP_ENOMEM, "optimiser state");
    c->ocfg = *o;
    int rc = launch_opt_reset(c);
    if (rc) return rc;
    c->have_opt = true;
    drop_graphs(c);  // the training graph bakes in the optimiser constants
    return NEP_OK;
}

int nep_optim_step(nep_ctx *c, const float *grad, const double *loss) {
    if (!c) return NEP_EINVAL;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (!c->have_params) return c->fail(NEP_ESTATE, "no parameters (call nep_set_params)");
    if (!grad) return c->fail(NEP_EINVAL, "null gradient");
    CK(cudaSetDevice(c->dev));
    int rc = launch_opt_step(c, grad, nullptr, 0.0, 0.0, 0.0, loss);
    if (rc) return rc;
    c->state_valid = false;
    return NEP_OK;
}

static int body_train(Ctx *c, double lE, double lF, double lV, double *loss3) {
    return body_loss(c, c->tgt_E.as<double>(), c->tgt_F.as<float>(), c->tgt_W.as<double>(),
                     c->tgt_has_hw ? c->tgt_hw.as<uint8_t>() : nullptr, lE, lF, lV, loss3, c->grad_int.as<float>(),
                     true);
}

int nep_train_step(nep_ctx *c, double lE, double lF, double lV, double *loss3) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (!c->have_targets) return c->fail(NEP_ESTATE, "no targets (call nep_set_targets)");
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (!std::isfinite(lE) || !std::isfinite(lF) || !std::isfinite(lV)) return c->fail(NEP_EINVAL, "non-finite weight");
    CK(cudaSetDevice(c->dev));
    double *l3 = loss3 ? loss3 : c->loss3_int.as<double>();
    if (c->schedule == NEP_SCHED_PLAIN) {
        rc = run_plain_loss(c, c->tgt_E.as<double>(), c->tgt_F.as<float>(), c->tgt_W.as<double>(),
                            c->tgt_has_hw ? c->tgt_hw.as<uint8_t>() : nullptr, lE, lF, lV, l3, c->grad_int.as<float>());
        if (!rc) rc = launch_opt_step(c, c->grad_int.as<float>(), l3, lE, lF, lV, nullptr);
    } else {
        uint64_t lb[3];
        std::memcpy(&lb[0], &lE, 8);
        std::memcpy(&lb[1], &lF, 8);
        std::memcpy(&lb[2], &lV, 8);
        std::vector<const void *> key = {l3, (const void *)(uintptr_t)lb[0], (const void *)(uintptr_t)lb[1],
                                         (const void *)(uintptr_t)lb[2]};
        rc = run_graph(c, c->g_train, key, [&] { return body_train(c, lE, lF, lV, l3); });
        c->last_timed = c->timing;
    }
    if (rc) return rc;
    c->state_valid = false;
    return NEP_OK;
}

int nep_optim_epoch_end(nep_ctx *c) {
    if (!c) return NEP_EINVAL;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    CK(cudaSetDevice(c->dev));
    return launch_opt_epoch(c);
}

int nep_optim_set_lr(nep_ctx *c, double lr) {
    if (!c) return NEP_EINVAL;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (!std::isfinite(lr) || !(lr > 0.0)) return c->fail(NEP_EINVAL, "learning rate must be finite and > 0");
    CK(cudaSetDevice(c->dev));
    return launch_opt_set_lr(c, lr);
}

int nep_optim_state(nep_ctx *c, double *out) {
    if (!c) return NEP_EINVAL;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (!out) return c->fail(NEP_EINVAL, "null output");
    CK(cudaSetDevice(c->dev));
    double st[OPT_NST];
    CK(cudaMemcpyAsync(st, c->opt_st.ptr, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out[0] = st[OPT_T];
    out[1] = st[OPT_LR];
    out[2] = st[OPT_BEST];
    out[3] = st[OPT_BAD];
    out[4] = st[OPT_LAST];
    out[5] = st[OPT_NRED];
    return NEP_OK;
}

int nep_get_params(nep_ctx *c, float *theta) {
    if (!c) return NEP_EINVAL;
    if (!c->have_params) return c->fail(NEP_ESTATE, "no parameters (call nep_set_params)");
    if (!theta) return c->fail(NEP_EINVAL, "null output");
    CK(cudaSetDevice(c->dev));
    if (c->P > 0) CK(cudaMemcpyAsync(theta, c->theta.ptr, sizeof(float) * c->P, cudaMemcpyDeviceToDevice, c->stream));
    return NEP_OK;
}

int nep_minibatch_setup(nep_ctx *c, int batch_size, int64_t *n_batches) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures (call nep_set_structures)");
    if (batch_size < 1) return c->fail(NEP_EINVAL, "batch size must be >= 1");
    CK(cudaSetDevice(c->dev));
    c->mb_var[0] = c->mb_var[1] = -1;
    int rc = build_minibatches(c, batch_size);
    if (rc) return rc;
    if ((rc = minibatch_tune(c))) return rc;
    c->state_valid = false;
    if (n_batches) *n_batches = (int64_t)c->mb.size();
    return NEP_OK;
}

static int mb_ready(nep_ctx *c, int64_t m) {
    int rc = ready(c);
    if (rc) return rc;
    if (c->mb_B < 1) return c->fail(NEP_ESTATE, "no mini-batches (call nep_minibatch_setup)");
    if (!c->have_targets) return c->fail(NEP_ESTATE, "no targets (call nep_set_targets)");
    if (m < 0 || m >= (int64_t)c->mb.size()) return c->fail(NEP_EINVAL, "mini-batch index out of range");
    return NEP_OK;
}

int nep_minibatch_loss_grad(nep_ctx *c, int64_t m, double lE, double lF, double lV, double *loss3, float *grad) {
    if (!c) return NEP_EINVAL;
    int rc = mb_ready(c, m);
    if (rc) return rc;
    if (!loss3 || !grad) return c->fail(NEP_EINVAL, "null output");
    if (!std::isfinite(lE) || !std::isfinite(lF) || !std::isfinite(lV)) return c->fail(NEP_EINVAL, "non-finite weight");
    CK(cudaSetDevice(c->dev));
    if ((rc = run_minibatch_loss(c, m, lE, lF, lV, loss3, grad))) return rc;
    c->state_valid = false;  // the per-atom state now holds one group only
    return NEP_OK;
}

static int mb_train_step(nep_ctx *c, int64_t m, double lE, double lF, double lV, double *loss3) {
    double *l3 = loss3 ? loss3 : c->loss3_int.as<double>();
    return run_minibatch_loss(c, m, lE, lF, lV, l3, c->grad_int.as<float>(), true);
}

int nep_minibatch_train_step(nep_ctx *c, int64_t m, double lE, double lF, double lV, double *loss3) {
    if (!c) return NEP_EINVAL;
    int rc = mb_ready(c, m);
    if (rc) return rc;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (!std::isfinite(lE) || !std::isfinite(lF) || !std::isfinite(lV)) return c->fail(NEP_EINVAL, "non-finite weight");
    CK(cudaSetDevice(c->dev));
    if ((rc = mb_train_step(c, m, lE, lF, lV, loss3))) return rc;
    c->state_valid = false;
    return NEP_OK;
}

int nep_minibatch_epoch(nep_ctx *c, const int64_t *order, int64_t n_steps, double lE, double lF, double lV) {
    if (!c) return NEP_EINVAL;
    int rc = mb_ready(c, 0);
    if (rc) return rc;
    if (!c->have_opt) return c->fail(NEP_ESTATE, "no optimiser (call nep_optim_init)");
    if (n_steps < 0 || (n_steps > 0 && !order)) return c->fail(NEP_EINVAL, "bad step list");
    if (!std::isfinite(lE) || !std::isfinite(lF) || !std::isfinite(lV)) return c->fail(NEP_EINVAL, "non-finite weight");
    for (int64_t k = 0; k < n_steps; ++k)
        if (order[k] < 0 || order[k] >= (int64_t)c->mb.size())
            return c->fail(NEP_EINVAL, "mini-batch index out of range");
    CK(cudaSetDevice(c->dev));
    // every group's training step is one cached graph, captured on its first step
    if ((rc = minibatch_shape_check(c))) return rc;
    uint64_t lb[3];
    std::memcpy(&lb[0], &lE, 8);
    std::memcpy(&lb[1], &lF, 8);
    std::memcpy(&lb[2], &lV, 8);
    if (c->mb_gkey != std::vector<uint64_t>(lb, lb + 3)) {
        drop_minibatch_graphs(c);
        c->mb_gkey.assign(lb, lb + 3);
    }
    if (c->mb_graphs.size() != c->mb.size()) c->mb_graphs.assign(c->mb.size(), nullptr);
    for (int64_t k = 0; k < n_steps; ++k) {
        cudaGraphExec_t &g = c->mb_graphs[order[k]];
        if (!g) {
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            rc = mb_train_step(c, order[k], lE, lF, lV, nullptr);
            const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return rc;
            }
            if (e != cudaSuccess) return c->fail_cuda(e, "cudaStreamEndCapture (mini-batch step)");
            const cudaError_t ei = cudaGraphInstantiate(&g, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                g = nullptr;
                return c->fail_cuda(ei, "cudaGraphInstantiate (mini-batch step)");
            }
        }
        CK(cudaGraphLaunch(g, c->stream));
    }
    c->state_valid = false;
    return launch_opt_epoch(c);
}

int nep_set_schedule(nep_ctx *c, int schedule) {
    if (!c) return NEP_EINVAL;
    if (schedule != NEP_SCHED_PERSISTENT && schedule != NEP_SCHED_PLAIN) return c->fail(NEP_EINVAL, "bad schedule");
    c->schedule = schedule;
    return NEP_OK;
}

int nep_get_launch(const nep_ctx *c, int *fw, int *fb, int *aw, int *ab) {
    if (!c) return NEP_EINVAL;
    if (fw) *fw = c->fwd.wpb;
    if (fb) *fb = c->fwd.blocks;
    if (aw) *aw = c->adj.wpb;
    if (ab) *ab = c->adj.blocks;
    return NEP_OK;
}

int nep_get_variant(const nep_ctx *c, int *fwd_lanes, int *fwd_regs, int *adj_lanes, int *adj_regs) {
    if (!c || !c->ks) return NEP_EINVAL;
    if (fwd_lanes) *fwd_lanes = c->ks->sw[c->fwd.var];
    if (fwd_regs) *fwd_regs = (c->fwd.var & 1) ? 96 : 128;
    if (adj_lanes) *adj_lanes = c->ks->sw[c->adj.var];
    if (adj_regs) *adj_regs = (c->adj.var & 1) ? 96 : 128;
    return NEP_OK;
}

int nep_set_variant(nep_ctx *c, int fwd_var, int adj_var) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures");
    if (fwd_var < 0 || fwd_var >= NVAR || adj_var < 0 || adj_var >= NVAR) return c->fail(NEP_EINVAL, "bad variant");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->stream));
    int rc;
    const int fw = std::min(c->fwd.wpb, c->ks->max_wpb[fwd_var]), aw = std::min(c->adj.wpb, c->ks->max_wpb[adj_var]);
    const int mf = max_blocks_per_sm(c, c->ks->fwd_fn[fwd_var], fw, c->ks->fwd_smem[fwd_var](c->T, c->NN) * fw);
    const int ma = max_blocks_per_sm(c, c->ks->adj_fn[adj_var], aw, c->ks->adj_smem[adj_var](c->T, c->NN) * aw);
    if (mf < 1 || ma < 1) return c->fail(NEP_EINVAL, "variant does not fit");
    if ((rc = make_sched(c, c->fwd, fw, c->n_sm * mf, fwd_var))) return rc;
    if ((rc = make_sched(c, c->adj, aw, c->n_sm * ma, adj_var))) return rc;
    if ((rc = alloc_sched_buffers(c))) return rc;
    drop_graphs(c);
    c->state_valid = false;
    return NEP_OK;
}

int nep_set_launch(nep_ctx *c, int fw, int fb, int aw, int ab) {
    if (!c) return NEP_EINVAL;
    if (!c->have_batch) return c->fail(NEP_ESTATE, "no structures");
    if (fw < 0 || fb < 0 || aw < 0 || ab < 0 || fw > 4 || aw > 4)
        return c->fail(NEP_EINVAL, "bad launch shape (at most 4 warps per block)");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->stream));
    int rc;
    fw = fw ? fw : c->fwd.wpb;
    aw = aw ? aw : c->adj.wpb;
    const int vf = c->fwd.var, va = c->adj.var;
    const int mf = max_blocks_per_sm(c, c->ks->fwd_fn[vf], fw, c->ks->fwd_smem[vf](c->T, c->NN) * fw);
    const int ma = max_blocks_per_sm(c, c->ks->adj_fn[va], aw, c->ks->adj_smem[va](c->T, c->NN) * aw);
    if (mf < 1 || ma < 1) return c->fail(NEP_EINVAL, "launch shape does not fit");
    fb = fb ? fb : c->n_sm * mf;
    ab = ab ? ab : c->n_sm * ma;
    if ((rc = make_sched(c, c->fwd, fw, fb, vf))) return rc;
    if ((rc = make_sched(c, c->adj, aw, ab, va))) return rc;
    if ((rc = alloc_sched_buffers(c))) return rc;
    drop_graphs(c);
    c->state_valid = false;
    return NEP_OK;
}

int nep_autotune(nep_ctx *c) {
    if (!c) return NEP_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    if (c->n_atoms == 0) return NEP_OK;
    CK(cudaSetDevice(c->dev));
    // cotangents for the adjoint timing: one pass with zero references and unit weights
    DevBuf zE, zF, zW, l3, gr;
    if (zE.ensure<double>(c->n_struct) || zF.ensure<float>(c->n_atoms * 3) || zW.ensure<double>(c->n_struct * 9) ||
        l3.ensure<double>(3) || gr.ensure<float>(c->P))
        return c->fail(NEP_ENOMEM, "autotune buffers");
    CK(cudaMemset(zE.ptr, 0, zE.bytes));
    CK(cudaMemset(zF.ptr, 0, zF.bytes));
    CK(cudaMemset(zW.ptr, 0, zW.bytes));
    const bool tsave = c->timing;
    c->timing = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_f = 1e30f, best_a = 1e30f;
    int bfw = c->fwd.wpb, bfb = c->fwd.blocks, bfv = c->fwd.var, baw = c->adj.wpb, bab = c->adj.blocks, bav = c->adj.var;
    const int wpbs[3] = {1, 2, 4};
    for (int var = 0; var < NVAR_TUNE && !rc; ++var) {
        for (int wpb : wpbs) {
            if (wpb > c->ks->max_wpb[var]) continue;
            const int mf = max_blocks_per_sm(c, c->ks->fwd_fn[var], wpb, c->ks->fwd_smem[var](c->T, c->NN) * wpb);
            const int ma = max_blocks_per_sm(c, c->ks->adj_fn[var], wpb, c->ks->adj_smem[var](c->T, c->NN) * wpb);
            for (int bps = 1; bps <= std::max(mf, ma); ++bps) {
                const bool tf = bps <= mf, ta = bps <= ma;
                if (tf && (rc = make_sched(c, c->fwd, wpb, c->n_sm * bps, var))) break;
                if (ta) {
                    if ((rc = make_sched(c, c->adj, wpb, c->n_sm * bps, var))) break;
                    if ((rc = alloc_sched_buffers(c))) break;
                }
                if ((rc = body_loss(c, zE.as<double>(), zF.as<float>(), zW.as<double>(), nullptr, 1.0, 1.0, 1.0,
                                    l3.as<double>(), gr.as<float>())))
                    break;
                float tbest_f = 1e30f, tbest_a = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    if (tf) {
                        CK(cudaEventRecord(e0, c->stream));
                        if ((rc = launch_forward(c, nullptr))) break;
                        CK(cudaEventRecord(e1, c->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        tbest_f = std::min(tbest_f, ms);
                    }
                    if (ta) {
                        CK(cudaEventRecord(e0, c->stream));
                        if ((rc = launch_adjoint(c))) break;
                        CK(cudaEventRecord(e1, c->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        tbest_a = std::min(tbest_a, ms);
                    }
                }
                if (rc) break;
                if (tf && tbest_f < best_f) {
                    best_f = tbest_f;
                    bfw = wpb;
                    bfb = c->n_sm * bps;
                    bfv = var;
                }
                if (ta && tbest_a < best_a) {
                    best_a = tbest_a;
                    baw = wpb;
                    bab = c->n_sm * bps;
                    bav = var;
                }
            }
            if (rc) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing = tsave;
    if (rc) return rc;
    if ((rc = make_sched(c, c->fwd, bfw, bfb, bfv))) return rc;
    if ((rc = make_sched(c, c->adj, baw, bab, bav))) return rc;
    if ((rc = alloc_sched_buffers(c))) return rc;
    drop_graphs(c);
    c->state_valid = false;
    CK(cudaStreamSynchronize(c->stream));
    return NEP_OK;
}

int nep_set_timing(nep_ctx *c, int on) {
    if (!c) return NEP_EINVAL;
    c->timing = on != 0;
    return NEP_OK;
}

int nep_kernel_times(nep_ctx *c, float *ms, int *n_io) {
    if (!c || !ms || !n_io) return NEP_EINVAL;
    if (!c->last_timed) return c->fail(NEP_ESTATE, "no timed call");
    const int n = std::min(*n_io, (int)KID_COUNT);
    CK(cudaEventSynchronize(c->ev[KID_COUNT]));
    for (int k = 0; k < n; ++k) CK(cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]));
    *n_io = n;
    return NEP_OK;
}

const char *nep_kernel_name(int k) { return (k >= 0 && k < KID_COUNT) ? kernel_names[k] : ""; }

const char *nep_last_error(const nep_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

