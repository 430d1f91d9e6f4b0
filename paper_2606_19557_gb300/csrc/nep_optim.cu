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

// Step counter and the powers beta^t (running products), and the epoch loss sum:
// L = lamE DE + lamF DF + lamV DV of this step when loss3 is given, else loss1[0].
__global__ void k_opt_tick(double *st, double b1, double b2, const double *loss3, double lE, double lF, double lV,
                           const double *loss1) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st[OPT_T] += 1.0;
        st[OPT_B1T] *= b1;
        st[OPT_B2T] *= b2;
        if (loss3) {
            st[OPT_ACC] += lE * loss3[0] + lF * loss3[1] + lV * loss3[2];
            st[OPT_NACC] += 1.0;
        } else if (loss1) {
            st[OPT_ACC] += loss1[0];
            st[OPT_NACC] += 1.0;
        }
    }
}

__global__ void k_amsgrad(int64_t P, float *__restrict__ theta, const float *__restrict__ g, double *__restrict__ m,
                          double *__restrict__ v, double *__restrict__ vmax, const double *__restrict__ st, double b1,
                          double b2, double eps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double bc1 = 1.0 - st[OPT_B1T], bc2 = 1.0 - st[OPT_B2T], lr = st[OPT_LR];
    const double gi = (double)g[i];
    const double mi = __dadd_rn(__dmul_rn(b1, m[i]), __dmul_rn(1.0 - b1, gi));
    const double vi = __dadd_rn(__dmul_rn(b2, v[i]), __dmul_rn(__dmul_rn(1.0 - b2, gi), gi));
    m[i] = mi;
    v[i] = vi;
    const double vh = vi / bc2;
    const double vm = vmax[i] > vh ? vmax[i] : vh;
    vmax[i] = vm;
    const double step = __dmul_rn(lr, mi / bc1) / __dadd_rn(sqrt(vm), eps);
    theta[i] = (float)__dadd_rn((double)theta[i], -step);
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

int launch_opt_step(Ctx *c, const float *grad, const double *loss3, double lE, double lF, double lV,
                    const double *loss1) {
    const nep_optim_config &o = c->ocfg;
    k_opt_tick<<<1, 32, 0, c->stream>>>(c->opt_st.as<double>(), o.beta1, o.beta2, loss3, lE, lF, lV, loss1);
    CK_LAUNCH("k_opt_tick");
    if (c->P > 0) {
        k_amsgrad<<<(unsigned)((c->P + 255) / 256), 256, 0, c->stream>>>(
            c->P, c->theta.as<float>(), grad, c->opt_m.as<double>(), c->opt_v.as<double>(), c->opt_vmax.as<double>(),
            c->opt_st.as<double>(), o.beta1, o.beta2, o.eps);
        CK_LAUNCH("k_amsgrad");
    }
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
