// Smoothed dual bound and its adjoint.
//
// For any positive output distribution q, max_x D(W_x || q) bounds C_n(d)
// from above (minimax form of the capacity; Sec. 2.3 reports the same
// quantity as the BA upper bound).  Parametrise q by one logit per output
// orbit class (Appendix A: optimal q is orbit-invariant),
//     q(c) = exp(theta[cls c]) / sum_c' exp(theta[cls c']),   L = log2 q,
// and smooth the max over inputs:
//     F(theta, d) = tau log2 sum_x 2^{D_x / tau},   max_x D_x <= F <= max_x D_x + tau n.
// With pi = softmax_x(D / tau) (in base 2) and W = b_k P_{n,k}:
//     dF/dL(c)        = -sum_x pi_x W(c|x) = -b_k (P_{n,k}^T pi)(c)    (a forward sweep of pi)
//     dF/dtheta_r     = (sum_{c in class r} dF/dL(c) + q(c)) / ln 2     (softmax chain; sum_c dF/dL = -1)
//     dF/dd (theta fixed) = sum_x pi_x sum_y rho_k W log2(W/q),  rho_k = (n-k)/d - k/(1-d)
//                     = sum_x pi_x [ sum_k rho_k b_k (log2 b_k - H_k(x)) - sum_y rho_k (b_k/C(n,k)) Count L ]
// (the last term is an adjoint sweep with weights rho_k b_k / C(n,k)).  The
// channel is never stored: D needs one adjoint sweep, the gradient one
// forward sweep, dF/dd a second adjoint sweep.
#include "bdc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int RT = 256;

template <typename T>
__global__ void k_theta_max(size_t M, const T *theta, const int32_t *cls, double *part, int slot) {
    __shared__ double red[RT / 32];
    double m = -INFINITY;
    for (size_t c = 1 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, (double)theta[cls[c]]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = -INFINITY;
        for (int w = 0; w < RT / 32; w++) t = fmax(t, red[w]);
        part[blockIdx.x * 4 + slot] = t;
    }
}

template <typename T>
__global__ void k_theta_sumexp(size_t M, const T *theta, const int32_t *cls, const double *inst_z, double *part) {
    __shared__ double red[RT / 32];
    const double mx = inst_z[I_DUAL_ZT];
    double s = 0.0;
    for (size_t c = 1 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x)
        s += exp((double)theta[cls[c]] - mx);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RT / 32; w++) t += red[w];
        part[blockIdx.x * 4 + 1] = t;
    }
}

// reductions of block partials into one instance slot
// op 0: max of part[b*4+slot] -> inst[dst]
// op 1: inst[dst] = inst[dst] + log(sum part[b*4+slot])       (log-sum-exp of theta)
// op 2: inst[dst] = sum part[b*4+slot]
// op 3: inst[dst] = 2 sum part[b*4+slot]    (a complement half of the inputs)
__global__ void k_fin(const double *part, int stride4, int nb, int slot, double *inst_z, int dst, int op) {
    __shared__ double red[FIN_THREADS / 32];
    double acc = (op == 0) ? fin_max(part + slot, stride4, nb, red) : fin_sum(part + slot, stride4, nb, red);
    if (threadIdx.x != 0) return;
    if (op == 1) inst_z[dst] = inst_z[dst] + log(acc);
    else inst_z[dst] = (op == 3) ? 2.0 * acc : acc;
}

template <typename T>
__global__ void k_make_L(size_t M, const T *theta, const int32_t *cls, const double *inst_z, T *L) {
    const double lse = inst_z[I_DUAL_ZT];
    const double inv_ln2 = 1.4426950408889634;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x)
        L[c] = (c == 0) ? (T)0 : (T)(((double)theta[cls[c]] - lse) * inv_ln2);
}

// sum_x 2^{(D_x - max)/tau}
__global__ void k_pi_sum(size_t N, const double *D, const double *inst_z, double tau, double *part) {
    __shared__ double red[RT / 32];
    const double mx = inst_z[I_DUAL_MAXD];
    double s = 0.0;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x)
        s += exp2((D[x] - mx) / tau);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RT / 32; w++) t += red[w];
        part[blockIdx.x * 4 + 0] = t;
    }
}

template <typename T>
__global__ void k_pi_write(size_t N, const double *D, double *inst_z, double tau, T *pd) {
    const double mx = inst_z[I_DUAL_MAXD], S = inst_z[I_DUAL_S];
    if (blockIdx.x == 0 && threadIdx.x == 0) inst_z[I_DUAL_F] = mx + tau * log2(S);
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x)
        pd[x] = (T)(exp2((D[x] - mx) / tau) / S);
}

// grad_theta[r] = sum over the codes of class r of (-b_k q_k^pi(c) + q(c)) / ln 2
template <typename T>
__global__ void k_grad_theta(int64_t Rout, const uint32_t *oreps, const T *qpi, const T *L, const double *bz,
                             T *grad) {
    const double inv_ln2 = 1.4426950408889634;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Rout; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t code = oreps[r];
        int k = bitlen32(code) - 1;
        uint32_t y = code ^ (1u << k);
        uint32_t mask = k ? ((1u << k) - 1u) : 0u;
        uint32_t ry = rev_bits(y, k);
        uint32_t mem[4] = {y, y ^ mask, ry, ry ^ mask};
        double acc = 0.0;
        for (int t = 0; t < 4; t++) {
            bool dup = false;
            for (int s = 0; s < t; s++) dup |= (mem[s] == mem[t]);
            if (dup) continue;
            uint32_t c = (1u << k) | mem[t];
            acc += -bz[k] * (double)qpi[c] + exp2((double)L[c]);
        }
        grad[r] = (T)(acc * inv_ln2);
    }
}

__global__ void k_activate_one(int nd, double *inst, int which, double tau) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < nd) inst[z * INST_STRIDE + I_ACTIVE] = (z == which) ? 1.0 : 0.0;
    if (z == which) inst[z * INST_STRIDE + I_DUAL_TAU] = tau;
}

int gridc(size_t n, int cap = 1024) {
    size_t g = (n + RT - 1) / RT;
    return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)cap));
}

template <typename T>
bdc_status dual_impl(bdc_engine *e, PrecBuf<T> &b, int z, const T *theta, double tau, double *F, double *maxD,
                     T *grad, double *grad_d) {
    const int n = e->n, nd = e->nd;
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    double *iz = e->inst + (size_t)z * INST_STRIDE;
    double *part0 = b.part + ((size_t)z * 2 + 0) * maxblk * 4;
    double *part1 = b.part + ((size_t)z * 2 + 1) * maxblk * 4;
    T *Lz = b.aux + z * M;
    const int gM = gridc(M), gN = gridc(N);
    k_activate_one<<<(nd + 63) / 64, 64, 0, e->stream>>>(nd, e->inst, z, tau); e->launches++;
    // log-sum-exp of theta over codes, then L = log2 softmax
    k_theta_max<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, part0, 0); e->launches++;
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part0, 4, gM, 0, iz, I_DUAL_ZT, 0); e->launches++;
    k_theta_sumexp<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, iz, part0); e->launches++;
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part0, 4, gM, 1, iz, I_DUAL_ZT, 1); e->launches++;
    k_make_L<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, iz, Lz); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    // q is constant on output classes, which are closed under complement, so
    // L(cpl c) = L(c) exactly and D(cpl x) = D(x): the sweeps run in the
    // complement half mode where the schedule allows, and D is mirrored
    const bool half = e->opt.use_half && half_possible(b.s);
    const int nbc = half ? b.s.nblk_cols / 2 : b.s.nblk_cols;
    // D_x for every input (double, into the spare array), block maxima
    BDC_TRY(sweep_adjoint<T>(e, b, b.aux, b.omega, reinterpret_cast<T *>(e->marg), MODE_DUAL, half));
    if (half) BDC_TRY(launch_mirror_half<double>(e, e->marg, b.s.n2));
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part1, 4, nbc, 1, iz, I_DUAL_MAXD, 0); e->launches++;
    const double *Dz = e->marg + z * N;
    k_pi_sum<<<gN, RT, 0, e->stream>>>(N, Dz, iz, tau, part0); e->launches++;
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part0, 4, gN, 0, iz, I_DUAL_S, 2); e->launches++;
    k_pi_write<T><<<gN, RT, 0, e->stream>>>(N, Dz, iz, tau, b.pd + z * N); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    if (grad) {
        // q_k^pi = P_{n,k}^T pi by the forward sweep (no BA update)
        BDC_TRY(sweep_forward<T>(e, b, b.pd, 0, MODE_DUAL, half));
        k_grad_theta<T><<<gridc((size_t)e->Rout), RT, 0, e->stream>>>(e->Rout, e->oreps, b.q + z * M, Lz,
                                                                       e->bk + (size_t)z * (n + 1), grad);
        e->launches++;
        BDC_CUDA_TRY(cudaGetLastError());
    }
    if (grad_d) {
        // sum_x pi_x (-Hb'(x) - G'(x)), Hb' = sum_k rho_k b_k H_k, G' with weights rho_k b_k / C(n,k)
        BDC_TRY(launch_build_Hb_w(e, e->dual_w, e->pcert));
        BDC_TRY(sweep_adjoint<T>(e, b, b.aux, b.omega2, reinterpret_cast<T *>(e->marg), MODE_DUAL_D, half));
        k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part1, 4, nbc, 0, iz, I_DUAL_GD, half ? 3 : 2); e->launches++;
        BDC_CUDA_TRY(cudaGetLastError());
    }
    std::vector<double> h(INST_STRIDE);
    BDC_CUDA_TRY(cudaMemcpyAsync(h.data(), iz, INST_STRIDE * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    cudaError_t err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        bdc_set_error(std::string("bdc_dual_bound: ") + cudaGetErrorString(err));
        return BDC_ECUDA;
    }
    if (F) *F = h[I_DUAL_F];
    if (maxD) *maxD = h[I_DUAL_MAXD];
    if (grad_d) *grad_d = h[I_DUAL_C0] + h[I_DUAL_GD];
    if (!std::isfinite(h[I_DUAL_F])) {
        bdc_set_error("bdc_dual_bound: non-finite value");
        return BDC_ENONFINITE;
    }
    return BDC_OK;
}

template <typename T>
__global__ void k_make_q(size_t M, const T *theta, const int32_t *cls, const double *inst_z, double *q) {
    const double lse = inst_z[I_DUAL_ZT];
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x)
        q[c] = (c == 0) ? 0.0 : exp((double)theta[cls[c]] - lse);
}

template <typename T>
bdc_status softmax_impl(bdc_engine *e, PrecBuf<T> &b, int z, const T *theta, double *q_out) {
    const size_t M = (size_t)2 << e->n;
    const int maxblk = part_maxblk(e);
    double *iz = e->inst + (size_t)z * INST_STRIDE;
    double *part0 = b.part + ((size_t)z * 2 + 0) * maxblk * 4;
    const int gM = gridc(M);
    k_theta_max<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, part0, 0); e->launches++;
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part0, 4, gM, 0, iz, I_DUAL_ZT, 0); e->launches++;
    k_theta_sumexp<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, iz, part0); e->launches++;
    k_fin<<<1, FIN_THREADS, 0, e->stream>>>(part0, 4, gM, 1, iz, I_DUAL_ZT, 1); e->launches++;
    k_make_q<T><<<gM, RT, 0, e->stream>>>(M, theta, e->ocls, iz, q_out); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    cudaError_t err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        bdc_set_error(std::string("bdc_softmax_classes: ") + cudaGetErrorString(err));
        return BDC_ECUDA;
    }
    return BDC_OK;
}

}  // namespace

extern "C" bdc_status bdc_softmax_classes(bdc_engine *e, int inst, const void *theta_dev, int prec, double *q_dev) {
    if (!e || !e->bound) {
        bdc_set_error("bdc_softmax_classes: no workspace bound");
        return BDC_ENOTBOUND;
    }
    if (inst < 0 || inst >= e->nd || !theta_dev || !q_dev || (prec != BDC_FP32 && prec != BDC_FP64)) {
        bdc_set_error("bdc_softmax_classes: bad arguments");
        return BDC_EINVAL;
    }
    if (prec == BDC_FP32) return softmax_impl<float>(e, e->f32, inst, (const float *)theta_dev, q_dev);
    return softmax_impl<double>(e, e->f64, inst, (const double *)theta_dev, q_dev);
}

extern "C" bdc_status bdc_dual_bound(bdc_engine *e, int inst, const void *theta_dev, double tau, int prec, double *F,
                                     double *max_D, void *grad_theta_dev, double *grad_d) {
    if (!e || !e->bound) {
        bdc_set_error("bdc_dual_bound: no workspace bound");
        return BDC_ENOTBOUND;
    }
    if (inst < 0 || inst >= e->nd || !theta_dev || !(tau > 0.0) || (prec != BDC_FP32 && prec != BDC_FP64)) {
        bdc_set_error("bdc_dual_bound: bad arguments (instance, theta, tau > 0, precision)");
        return BDC_EINVAL;
    }
    if (grad_d && !(e->d[inst] > 0.0 && e->d[inst] < 1.0)) {
        bdc_set_error("bdc_dual_bound: dF/dd needs a BDC_d instance with 0 < d < 1 (not a length mixture)");
        return BDC_EINVAL;
    }
    if (prec == BDC_FP32)
        return dual_impl<float>(e, e->f32, inst, (const float *)theta_dev, tau, F, max_D, (float *)grad_theta_dev,
                                grad_d);
    return dual_impl<double>(e, e->f64, inst, (const double *)theta_dev, tau, F, max_D, (double *)grad_theta_dev,
                             grad_d);
}

namespace {

// theta[r] = ln max(q(rep_r), floor): logits whose softmax over classes is q
// for an orbit-invariant q normalised to 1 (the inverse of the expansion)
template <typename T>
__global__ void k_class_logits(int64_t Rout, const uint32_t *oreps, const double *q, double floor_v, T *theta) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Rout; r += (int64_t)gridDim.x * blockDim.x)
        theta[r] = (T)log(fmax(q[oreps[r]], floor_v));
}

}  // namespace

extern "C" bdc_status bdc_class_logits(bdc_engine *e, const double *q_dev, double floor_v, int prec,
                                       void *theta_dev) {
    if (!e || !e->bound) {
        bdc_set_error("bdc_class_logits: no workspace bound");
        return BDC_ENOTBOUND;
    }
    if (!q_dev || !theta_dev || !(floor_v > 0.0) || (prec != BDC_FP32 && prec != BDC_FP64)) {
        bdc_set_error("bdc_class_logits: bad arguments (q, theta, floor > 0, precision)");
        return BDC_EINVAL;
    }
    const int g = (int)std::min<int64_t>((e->Rout + RT - 1) / RT, 4096);
    if (prec == BDC_FP32)
        k_class_logits<float><<<g, RT, 0, e->stream>>>(e->Rout, e->oreps, q_dev, floor_v, (float *)theta_dev);
    else
        k_class_logits<double><<<g, RT, 0, e->stream>>>(e->Rout, e->oreps, q_dev, floor_v, (double *)theta_dev);
    e->launches++;
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        bdc_set_error(std::string("bdc_class_logits: ") + cudaGetErrorString(err));
        return BDC_ECUDA;
    }
    return BDC_OK;
}
