// Mini-batch mode (Sec. "Training": each optimisation step uses a mini-batch of
// structures; the geometry-dependent data are built once and kept on the GPU).
//
// The cached batch is split into groups of `batch_size` consecutive structures.  A
// group is a contiguous range of structures and atoms, so the neighbour lists, the
// pair records and the per-atom buffers of the whole batch serve every group as they
// are: only the schedules differ.  For each group the host builds, once:
//   * its work order (its atoms sorted by species, at work positions [a0, a1));
//   * cost-balanced warp ranges for the forward and adjoint kernels, with as many warps
//     as the group fills (one batch of atoms per warp when it is small);
//   * the species runs of the adjoint warps and the network-gradient chunks.
// A step then launches the same kernels as the whole-batch pass on those slices, with
// the group's own normalisers N_s, N_a and N_s^V in Eq. "loss".
#include <algorithm>
#include <numeric>
#include <vector>

#include "nep_ctx.cuh"

namespace nep {

namespace {

// Cost-balanced split of the positions [p0, p1) (prefix costs pre, relative to p0) over W
// warps; returns W + 1 global boundaries.
std::vector<int> split_warps(const std::vector<double> &pre, int p0, int W) {
    const int n = (int)pre.size() - 1;
    std::vector<int> begin(W + 1, p0 + n);
    const double tot = pre[n];
    int q = 0;
    for (int w = 0; w < W; ++w) {
        const double target = tot * (double)w / (double)W;
        while (q < n && pre[q] < target) ++q;
        begin[w] = p0 + q;
    }
    for (int w = 1; w <= W; ++w) begin[w] = std::max(begin[w], begin[w - 1]);
    return begin;
}

// First and last warp (relative to the launch) holding positions of each species.
void species_warps(const std::vector<int> &begin, const std::vector<int> &tb /*[T+1] global*/, int T, int *wlo,
                   int *whi) {
    const int W = (int)begin.size() - 1;
    auto owner = [&](int p) {
        int lo = 0, hi = W - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (begin[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    for (int t = 0; t < T; ++t) {
        wlo[t] = 0;
        whi[t] = -1;
        if (tb[t + 1] > tb[t]) {
            wlo[t] = owner(tb[t]);
            whi[t] = owner(tb[t + 1] - 1);
        }
    }
}

void shape_key(const Ctx *c, int *key) {
    key[0] = c->fwd.var;
    key[1] = c->fwd.wpb;
    key[2] = c->fwd.W;
    key[3] = c->adj.var;
    key[4] = c->adj.wpb;
    key[5] = c->adj.W;
    key[0] += 16 * (c->mb_var[0] + 1);  // the group variants, when set, change the schedules too
    key[3] += 16 * (c->mb_var[1] + 1);
}

// Variant and warps per block of the group launches: the chosen group variant with the
// largest block its launch bounds allow, else the batch's own shape.
void group_launch(const Ctx *c, int which, int &var, int &wpb, int &wcap) {
    const Sched &s = which == 0 ? c->fwd : c->adj;
    const int v = c->mb_var[which];
    if (v < 0) {
        var = s.var;
        wpb = s.wpb;
        wcap = s.W;
    } else {
        var = v;
        // the largest block the launch bounds allow that fits the shared-memory budget
        const void *fn = which == 0 ? c->ks->fwd_fn[v] : c->ks->adj_fn[v];
        wpb = 1;
        for (int w = c->ks->max_wpb[v]; w >= 1; w /= 2) {
            const size_t sm = (which == 0 ? c->ks->fwd_smem[v] : c->ks->adj_smem[v])(c->T, c->NN) * w;
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, w * 32, sm) != cudaSuccess) cudaGetLastError();
            if (nb >= 1) {
                wpb = w;
                break;
            }
        }
        // adjoint warps write per-warp gradient slots sized for the batch's adjoint grid
        wcap = which == 0 ? c->n_sm * 16 : c->adj.W / wpb * wpb;
    }
}

}  // namespace

void drop_minibatch_graphs(Ctx *c) {
    for (cudaGraphExec_t g : c->mb_graphs)
        if (g) cudaGraphExecDestroy(g);
    c->mb_graphs.clear();
    c->mb_gkey.clear();
}

int minibatch_shape_check(Ctx *c) {
    int key[6];
    shape_key(c, key);
    return std::equal(key, key + 6, c->mb_key) ? NEP_OK : build_minibatches(c, c->mb_B);
}

int build_minibatches(Ctx *c, int B) {
    drop_minibatch_graphs(c);  // the graphs hold the old schedules
    if (int rc = fetch_host_lists(c)) return rc;
    const int64_t ns = c->n_struct, na = c->n_atoms;
    const int T = c->T;
    int fvar, fwpb, fcap, avar, awpb, acap;
    group_launch(c, 0, fvar, fwpb, fcap);
    group_launch(c, 1, avar, awpb, acap);
    const int gf = 32 / c->ks->sw[fvar], ga = 32 / c->ks->sw[avar];
    std::vector<int> work(na);
    std::vector<int> wbf, wba, wlo, whi, chunks, clo, chi;
    std::vector<Ctx::MiniBatch> mbs;
    for (int64_t s0 = 0; s0 < ns; s0 += B) {
        Ctx::MiniBatch m{};
        m.s0 = s0;
        m.s1 = std::min<int64_t>(ns, s0 + B);
        m.a0 = c->h_atom_off[m.s0];
        m.a1 = c->h_atom_off[m.s1];
        const int p0 = (int)m.a0, n = (int)(m.a1 - m.a0);
        // work order: the group's atoms by species (stable)
        for (int k = 0; k < n; ++k) work[p0 + k] = p0 + k;
        std::stable_sort(work.begin() + p0, work.begin() + p0 + n,
                         [&](int x, int y) { return c->h_type[x] < c->h_type[y]; });
        std::vector<int> tb(T + 1, p0);
        for (int k = 0; k < n; ++k) tb[c->h_type[work[p0 + k]] + 1]++;
        for (int t = 0; t < T; ++t) tb[t + 1] += tb[t] - p0;
        std::vector<double> pre(n + 1, 0.0);
        for (int k = 0; k < n; ++k) {
            const int i = work[p0 + k];
            pre[k + 1] = pre[k] + (double)(c->h_nbr_off[i + 1] - c->h_nbr_off[i]) + 6.0 * c->h_nang[i] + 8.0;
        }
        // warps: one batch of atoms each for a small group, at most the full persistent grid
        auto warps = [&](int g, int wpb, int cap) {
            int W = std::max(1, (n + g - 1) / g);
            W = std::min(W, cap);
            return (W + wpb - 1) / wpb * wpb;
        };
        m.Wf = warps(gf, fwpb, fcap);
        m.Wa = warps(ga, awpb, acap);
        const std::vector<int> bf = split_warps(pre, p0, m.Wf), ba = split_warps(pre, p0, m.Wa);
        m.wf_off = (int64_t)wbf.size();
        wbf.insert(wbf.end(), bf.begin(), bf.end());
        m.wa_off = (int64_t)wba.size();
        wba.insert(wba.end(), ba.begin(), ba.end());
        const size_t tofs = wlo.size();
        wlo.resize(tofs + T);
        whi.resize(tofs + T);
        species_warps(ba, tb, T, wlo.data() + tofs, whi.data() + tofs);
        // network chunks of one species each: about one per SM in a small group (the network
        // kernels run one block per chunk), 128 work positions at most
        const int CH = std::max(16, std::min(128, n / std::max(1, c->n_sm) / 16 * 16));
        m.ch = CH;
        m.ck_off = (int64_t)chunks.size();
        clo.resize(tofs + T);
        chi.resize(tofs + T);
        for (int t = 0; t < T; ++t) {
            clo[tofs + t] = (int)(chunks.size() - m.ck_off);
            for (int p = tb[t]; p < tb[t + 1]; p += CH) chunks.push_back(p);
            chi[tofs + t] = (int)(chunks.size() - m.ck_off);
        }
        m.n_ck = (int)(chunks.size() - m.ck_off);
        chunks.push_back((int)m.a1);
        mbs.push_back(m);
    }
    const int64_t nm = (int64_t)mbs.size();
    int max_ck = 0;
    for (const Ctx::MiniBatch &m : mbs) max_ck = std::max(max_ck, m.n_ck);
    const size_t arow = sizeof(float) * (size_t)(c->NN * c->NDP + 2 * c->NN);
    if (c->annpart.bytes < arow * (size_t)(max_ck + 1)) {
        drop_graphs(c);  // the whole-batch graphs hold the old partial buffer
        if (c->annpart.ensure_bytes(arow * (size_t)(max_ck + 1))) return c->fail(NEP_ENOMEM, "network partials");
    }
    if (c->mb_work.ensure<int>(std::max<int64_t>(na, 1)) || c->mb_wbf.ensure<int>((int64_t)wbf.size() + 1) ||
        c->mb_wba.ensure<int>((int64_t)wba.size() + 1) || c->mb_wlo.ensure<int>(nm * T + 1) ||
        c->mb_whi.ensure<int>(nm * T + 1) || c->mb_chunks.ensure<int>((int64_t)chunks.size() + 1) ||
        c->mb_clo.ensure<int>(nm * T + 1) || c->mb_chi.ensure<int>(nm * T + 1))
        return c->fail(NEP_ENOMEM, "mini-batch schedules");
    auto up = [&](DevBuf &d, const std::vector<int> &h) {
        return h.empty() ? cudaSuccess : cudaMemcpy(d.ptr, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
    };
    CK(up(c->mb_work, work));
    if (int rc = build_work_rec(c, c->mb_work.as<int>(), c->mb_rec, c->mb_rec2)) return rc;
    CK(up(c->mb_wbf, wbf));
    CK(up(c->mb_wba, wba));
    CK(up(c->mb_wlo, wlo));
    CK(up(c->mb_whi, whi));
    CK(up(c->mb_chunks, chunks));
    CK(up(c->mb_clo, clo));
    CK(up(c->mb_chi, chi));
    c->mb = std::move(mbs);
    c->mb_B = B;
    c->mb_used[0] = fvar;
    c->mb_used[1] = fwpb;
    c->mb_used[2] = avar;
    c->mb_used[3] = awpb;
    shape_key(c, c->mb_key);
    return NEP_OK;
}

// Small groups leave most of the GPU idle, and the fastest kernel variant is then often not
// the batch's one (16 lanes per atom halve the atoms, so the latency, of a warp's batch):
// time a loss + gradient pass over the first groups for a few variant pairs, keep the
// fastest.  Needs parameters and targets; otherwise the batch's own variants stay.
int minibatch_tune(Ctx *c) {
    if (!c->have_targets || !c->have_params || c->mb.empty()) return NEP_OK;
    const int cand[][2] = {{-1, -1}, {2, 2}, {3, 2}, {3, 3}, {0, 0}, {4, 4}, {5, 5}, {4, 5}};
    const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    const int ng = (int)std::min<size_t>(8, c->mb.size());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bi = 0, rc = NEP_OK;
    for (int k = 0; k < ncand && !rc; ++k) {
        c->mb_var[0] = cand[k][0];
        c->mb_var[1] = cand[k][1];
        if ((rc = build_minibatches(c, c->mb_B))) break;
        float ms = 0.0f;
        int trc = NEP_OK;  // a candidate that cannot launch (too large a model) is skipped
        for (int rep = 0; rep < 2 && !trc; ++rep) {  // the first repetition warms up
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) trc = NEP_ECUDA;
            for (int m = 0; m < ng && !trc; ++m)
                trc = run_minibatch_loss(c, m, 1.0, 1.0, 0.1, c->loss3_int.as<double>(), c->grad_int.as<float>());
            if (!trc && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                trc = NEP_ECUDA;
        }
        if (trc) {
            cudaStreamSynchronize(c->stream);
            cudaGetLastError();
            continue;
        }
        if (ms < best) {
            best = ms;
            bi = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->mb_var[0] = cand[bi][0];
    c->mb_var[1] = cand[bi][1];
    return build_minibatches(c, c->mb_B);
}

// Loss and gradient of group m against the references of nep_set_targets.  The padded
// parameter copies are current (nep_set_params expands them, every optimiser update
// refreshes them), so the step starts with the descriptors.
int run_minibatch_loss(Ctx *c, int64_t mi, double lE, double lF, double lV, double *loss3, float *grad, bool opt) {
    int rc0 = minibatch_shape_check(c);  // the launch shape may have changed since the setup
    if (rc0) return rc0;
    const Ctx::MiniBatch &m = c->mb[mi];
    const int T = c->T;
    const uint8_t *hw = c->tgt_has_hw ? c->tgt_hw.as<uint8_t>() : nullptr;
    // the group's own normalisers (restored below: they only enter launch arguments)
    const double sNs = c->ov_Ns, sNa = c->ov_Na, sNsV = c->ov_NsV;
    c->ov_Ns = (double)(m.s1 - m.s0);
    c->ov_Na = (double)(m.a1 - m.a0);
    c->ov_NsV = 0.0;
    int rc = NEP_OK;
    do {
        if ((rc = launch_forward_sched(c, c->mb_work.as<int>(), c->mb_rec, c->mb_rec2, c->mb_wbf.as<int>() + m.wf_off,
                                       m.Wf / c->mb_used[1],
                                       c->mb_used[0], c->mb_used[1], c->mb_chunks.as<int>() + m.ck_off, m.n_ck,
                                       m.ch)))
            break;
        TermsCall t;
        t.a0 = m.a0;
        t.a1 = m.a1;
        t.s0 = m.s0;
        t.s1 = m.s1;
        t.F_out = c->F_int.as<float>();
        t.E_out = c->E_int.as<double>();
        t.W_out = c->W_int.as<double>();
        t.loss = true;
        t.F_ref = c->tgt_F.as<float>();
        t.E_ref = c->tgt_E.as<double>();
        t.W_ref = c->tgt_W.as<double>();
        t.has_W = hw;
        t.lE = lE;
        t.lF = lF;
        t.lV = lV;
        t.nsv = host_nsv(c, hw, m.s0, m.s1);
        t.loss3 = loss3;
        if ((rc = launch_terms(c, t))) break;
        if ((rc = launch_adjoint_sched(c, c->mb_work.as<int>(), c->mb_rec, c->mb_rec2, c->mb_wba.as<int>() + m.wa_off,
                                       m.Wa / c->mb_used[3],
                                       c->mb_used[2], c->mb_used[3], c->mb_chunks.as<int>() + m.ck_off, m.n_ck,
                                       m.ch)))
            break;
        if ((rc = launch_ann_grad_chunks(c, c->mb_chunks.as<int>() + m.ck_off, m.n_ck))) break;
        rc = launch_grad_final_sched(c, grad, c->mb_clo.as<int>() + mi * T, c->mb_chi.as<int>() + mi * T,
                                     c->mb_wlo.as<int>() + mi * T, c->mb_whi.as<int>() + mi * T,
                                     c->mb_wba.as<int>() + m.wa_off, opt, loss3, lE, lF, lV);
    } while (0);
    c->ov_Ns = sNs;
    c->ov_Na = sNa;
    c->ov_NsV = sNsV;
    return rc;
}

}  // namespace nep
