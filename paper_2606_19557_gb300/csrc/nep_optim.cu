// Optimiser of the training loop (Sec. "Training"): Adam with the AMSGrad variant and
// the epoch-level plateau schedule, on the device so that training steps replay as one
// CUDA graph with no host round trip.
//
//   m_t = beta1 m_{t-1} + (1 - beta1) g_t,   v_t = beta2 v_{t-1} + (1 - beta2) g_t^2
//   m^_t = m_t / (1 - beta1^t),              v^_t = v_t / (1 - beta2^t)
//   v^max_t = max(v^max_{t-1}, v^_t)         (maximum of the bias-corrected moment)
//   theta_t = theta_{t-1} - eta m^_t / (sqrt(v^max_t) + eps)
//   eta_{e+1} = max(gamma eta_e, eta_min) after p consecutive epochs whose mean loss
//   did not improve on the best one by the relative threshold tau.
//
// Parameters stay FP32 (the precision of the pass); moments and update arithmetic are
// FP64.  The P-element update is a few tens of kilobytes: one short elementwise launch.
#include <math_constants.h>

#include <algorithm>

#include "nep_ctx.cuh"

namespace nep {

namespace {

__global__ void k_opt_reset(double *st, double lr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st[OPT_T] = 0.0;
        st[OPT_B1T] = 1.0;
        st[OPT_B2T] = 1.0;
        st[OPT_LR] = lr;
        st[OPT_BEST] = CUDART_INF;
        st[OPT_BAD] = 0.0;
        st[OPT_ACC] = 0.0;
        st[OPT_NACC] = 0.0;
        st[OPT_LAST] = CUDART_NAN;
        st[OPT_NRED] = 0.0;
    }
}

__global__ void k_opt_set_lr(double *st, double lr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st[OPT_LR] = lr;
        st[OPT_BEST] = CUDART_INF;
        st[OPT_BAD] = 0.0;
    }
}

// One AMSGrad step over the P parameters (the padded copies follow each update); the
// block that finishes last advances the step counter, the powers beta^t and the epoch loss
// sum (L = lamE DE + lamF DF + lamV DV of this step when loss3 is given, else loss1[0]).
__global__ void k_opt_step(int64_t P, const float *__restrict__ g, OptArgs o, unsigned *counter) {
    grid_dep_wait();
    grid_dep_launch();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const OptStep s = opt_step_state(o);
    if (i < P) amsgrad_elem(o, s, i, (double)g[i]);
    if (last_block_arrival(counter, gridDim.x, false) && threadIdx.x == 0) opt_tick(o);
}

// Epoch boundary: mean loss of the epoch's steps, improvement test, rate reduction.
__global__ void k_opt_epoch(double *st, double factor, double patience, double lr_min, double thr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (st[OPT_NACC] > 0.0) {
            const double L = st[OPT_ACC] / st[OPT_NACC];
            st[OPT_LAST] = L;
            if (L < st[OPT_BEST] * (1.0 - thr)) {
                st[OPT_BEST] = L;
                st[OPT_BAD] = 0.0;
            } else {
                st[OPT_BAD] += 1.0;
            }
            if (st[OPT_BAD] >= patience) {
                const double r = factor * st[OPT_LR];
                st[OPT_LR] = r > lr_min ? r : lr_min;
                st[OPT_BAD] = 0.0;
                st[OPT_NRED] += 1.0;
            }
        }
        st[OPT_ACC] = 0.0;
        st[OPT_NACC] = 0.0;
    }
}

}  // namespace

int launch_opt_reset(Ctx *c) {
    CK(cudaMemsetAsync(c->opt_m.ptr, 0, sizeof(double) * c->P, c->stream));
    CK(cudaMemsetAsync(c->opt_v.ptr, 0, sizeof(double) * c->P, c->stream));
    CK(cudaMemsetAsync(c->opt_vmax.ptr, 0, sizeof(double) * c->P, c->stream));
    k_opt_reset<<<1, 32, 0, c->stream>>>(c->opt_st.as<double>(), c->ocfg.lr);
    CK_LAUNCH("k_opt_reset");
    return NEP_OK;
}

int launch_opt_set_lr(Ctx *c, double lr) {
    k_opt_set_lr<<<1, 32, 0, c->stream>>>(c->opt_st.as<double>(), lr);
    CK_LAUNCH("k_opt_set_lr");
    return NEP_OK;
}

ParScatter par_scatter(Ctx *c) {
    ParScatter p;
    p.po = c->po;
    p.T = c->T;
    p.NN = c->NN;
    p.ND = c->ND;
    p.NDP = c->NDP;
    p.nR = c->nR;
    p.kR = c->kR;
    p.nA = c->nA;
    p.kA = c->kA;
    p.NRP = c->ks->NR;
    p.KRP = c->ks->KR;
    p.NAP = c->ks->NA;
    p.KAP = c->ks->KA;
    p.map = c->d_desc_map.as<int>();
    p.par = c->par.as<float>();
    return p;
}

OptArgs opt_args(Ctx *c, const double *loss3, double lE, double lF, double lV, const double *loss1) {
    const nep_optim_config &cf = c->ocfg;
    OptArgs o;
    o.theta = c->theta.as<float>();
    o.m = c->opt_m.as<double>();
    o.v = c->opt_v.as<double>();
    o.vmax = c->opt_vmax.as<double>();
    o.st = c->opt_st.as<double>();
    o.b1 = cf.beta1;
    o.b2 = cf.beta2;
    o.eps = cf.eps;
    o.loss3 = loss3;
    o.lE = lE;
    o.lF = lF;
    o.lV = lV;
    o.loss1 = loss1;
    o.ps = par_scatter(c);
    return o;
}

int launch_opt_step(Ctx *c, const float *grad, const double *loss3, double lE, double lF, double lV,
                    const double *loss1) {
    const unsigned nb = (unsigned)std::max<int64_t>(1, (c->P + 255) / 256);
    CK(launch_k(c->pdl(), k_opt_step, nb, 256, 0, c->stream, c->P, grad, opt_args(c, loss3, lE, lF, lV, loss1),
                c->counters.as<unsigned>() + 1));
    return NEP_OK;
}

int launch_opt_epoch(Ctx *c) {
    const nep_optim_config &o = c->ocfg;
    k_opt_epoch<<<1, 32, 0, c->stream>>>(c->opt_st.as<double>(), o.factor, (double)o.patience, o.lr_min,
                                         o.threshold);
    CK_LAUNCH("k_opt_epoch");
    return NEP_OK;
}

}  // namespace nep
