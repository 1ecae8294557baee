// Level-by-level sweep through global memory: the schedule for sizes whose
// tiles do not fit in shared memory (FP64 at n >= 27: a row tile of the
// split schedule would need 2^15 doubles, 256 KB).  The same recursion as the
// tiled passes, one input symbol per launch, every level a full array of
// 2^(n+1) values in HBM (two ping-pong buffers):
//
//   forward (d-free: embedding counts), level i -> i+1, index P = (code(u) << (n-i)) | s:
//     F_{i+1}(u, s') = F_i(u, 0 s') + F_i(u, 1 s')   [|u| <= i]
//                    + F_i(u^-, u_last s')            [|u| >= 1]
//   from F_0(empty, x) = p(x) to F_n(y) = sum_x p(x) Count(y, x) = C(n,k) q_k(y);
//   adjoint, level i+1 -> i:
//     Gbar_i(v, b s') = Gbar_{i+1}(v, s') + Gbar_{i+1}(v b, s')
//   from Gbar_n(y) = omega_{|y|} L(y) to G(x) = Gbar_0(empty, x).
//
// Each level reads about three values and writes one per element: 2^(n+1)
// (4 + 4) bytes at FP64 per level, n levels per sweep (n = 28: 240 GB, tens
// of milliseconds), which is what a once-per-run certificate can afford.
// Every addition adds same-sign terms, one (adjoint) or two (forward) per
// level, so the rounding analysis of the tiled sweep carries over: a path of
// the adjoint from L(y) to G(x) passes through n additions.
#include "bdc_internal.cuh"

#include <algorithm>

namespace {

constexpr int ST_THREADS = 256;

// level 0: A[(1 << n) | x] = p(x) (after the pending BA update where asked),
// every other slot 0; block sums of p into part slot 0 (exactly nb blocks)
template <typename T>
__global__ void k_stream_init_fwd(int n, T *p, const T *D, T *A, double *part, int maxblk, double *inst,
                                  int apply_update) {
    __shared__ double red[ST_THREADS / 32];
    const int z = blockIdx.y;
    const double *I = inst + z * INST_STRIDE;
    if (!flag_set(I, I_ACTIVE)) return;
    const size_t N = (size_t)1 << n, M = N << 1;
    T *pz = p + z * N;
    const T *Dz = D + z * N;
    T *Az = A + z * M;
    const bool upd = apply_update && flag_set(I, I_PENDING);
    const T sh = (T)I[I_SHIFT];
    double s = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x) {
        if (!BDC_IN_RANGE(c, M, I)) continue;
        if (c < N) {
            Az[c] = (T)0;
        } else {
            T v = pz[c - N];
            if (upd) {
                v = v * exp2_t<T>(Dz[c - N] - sh);
                pz[c - N] = v;
            }
            Az[c] = v;
            s += (double)v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < ST_THREADS / 32; w++) t += red[w];
        part[((size_t)z * 2 + 0) * maxblk * 4 + blockIdx.x * 4] = t;
    }
}

// forward level i -> i+1 (rest = n - i - 1 pending symbols after it)
template <typename T>
__global__ void k_stream_fwd(int n, int i, const T *__restrict__ A, T *__restrict__ B, const double *inst) {
    const int z = blockIdx.y;
    if (!flag_set(inst + z * INST_STRIDE, I_ACTIVE)) return;
    const size_t M = (size_t)2 << n;
    const T *Az = A + z * M;
    T *Bz = B + z * M;
    const int rest = n - i - 1;
    const size_t smask = ((size_t)1 << rest) - 1;
    for (size_t P = (size_t)blockIdx.x * blockDim.x + threadIdx.x; P < M; P += (size_t)gridDim.x * blockDim.x) {
        const size_t cu = P >> rest, s = P & smask;
        T v = (T)0;
        if (cu != 0) {
            const int k = 63 - __clzll((long long)cu);  // |u|
            if (k <= i) {
                const size_t base = (cu << (rest + 1)) | s;
                if (BDC_IN_RANGE(base | ((size_t)1 << rest), M, inst + z * INST_STRIDE))
                    v = Az[base] + Az[base | ((size_t)1 << rest)];
            }
            const size_t j = ((cu >> 1) << (rest + 1)) | ((cu & 1u) << rest) | s;
            if (k >= 1 && BDC_IN_RANGE(j, M, inst + z * INST_STRIDE)) v = v + Az[j];
        }
        Bz[P] = v;
    }
}

// q_k(y) = F_n(y) / C(n,k) and its log (floored in iterations, capped at 1 in
// the certificate, like the tiled passes)
template <typename T>
__global__ void k_stream_q(int n, const T *F, T *q, T *L, const double *inv_binom, double q_floor, int mode,
                           const double *inst) {
    const int z = blockIdx.y;
    if (!flag_set(inst + z * INST_STRIDE, I_ACTIVE)) return;
    const size_t M = (size_t)2 << n;
    const T *Fz = F + z * M;
    T *qz = q + z * M, *Lz = L + z * M;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x) {
        if (c == 0) {
            qz[0] = (T)0;
            Lz[0] = (T)0;
            continue;
        }
        const int k = 63 - __clzll((long long)c);
        const T qv = Fz[c] * (T)inv_binom[k];
        qz[c] = qv;
        Lz[c] = log2_t<T>(mode == MODE_CERT ? (qv < (T)1 ? qv : (T)1) : (qv > (T)q_floor ? qv : (T)q_floor));
    }
}

// adjoint level n: omega_k L(y) at every code
template <typename T>
__global__ void k_stream_init_adj(int n, const T *Lsrc, const T *omega, T *A, const double *inst) {
    const int z = blockIdx.y;
    if (!flag_set(inst + z * INST_STRIDE, I_ACTIVE)) return;
    const size_t M = (size_t)2 << n;
    const T *Lz = Lsrc + z * M;
    const T *om = omega + z * (n + 1);
    T *Az = A + z * M;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x)
        Az[c] = c ? om[63 - __clzll((long long)c)] * Lz[c] : (T)0;
}

// adjoint level i+1 -> i (rest = n - i - 1: the index at level i is
// (code(v) << (rest + 1)) | (b << rest) | s')
template <typename T>
__global__ void k_stream_adj(int n, int i, const T *__restrict__ A, T *__restrict__ B, const double *inst) {
    const int z = blockIdx.y;
    if (!flag_set(inst + z * INST_STRIDE, I_ACTIVE)) return;
    const size_t M = (size_t)2 << n;
    const T *Az = A + z * M;
    T *Bz = B + z * M;
    const int rest = n - i - 1;
    const size_t smask = ((size_t)1 << rest) - 1;
    for (size_t P = (size_t)blockIdx.x * blockDim.x + threadIdx.x; P < M; P += (size_t)gridDim.x * blockDim.x) {
        const size_t cv = P >> (rest + 1), b = (P >> rest) & 1u, s = P & smask;
        T v = (T)0;
        const size_t j1 = (cv << rest) | s, j2 = (((cv << 1) | b) << rest) | s;
        if (cv != 0 && cv < ((size_t)2 << i) && BDC_IN_RANGE(j1, M, inst + z * INST_STRIDE) &&
            BDC_IN_RANGE(j2, M, inst + z * INST_STRIDE))
            v = Az[j1] + Az[j2];
        Bz[P] = v;
    }
}

// the epilogue of the tiled adjoint columns pass, per input x, from
// G(x) = Gbar_0 at (1 << n) | x; block partials into part slot 1 (exactly nb blocks)
template <typename T>
__global__ void k_stream_epi(int n, const T *Gl, const T *Hb, const T *p, void *Dout, const double *hb2, double *part,
                             int maxblk, const double *inst, int mode, double eH_scale, double u) {
    __shared__ double red[ST_THREADS / 32];
    const int z = blockIdx.y;
    const double *I = inst + z * INST_STRIDE;
    if (!flag_set(I, I_ACTIVE)) return;
    const size_t N = (size_t)1 << n;
    const T *Gz = Gl + z * (N << 1) + N;
    const T *Hbz = Hb + z * N;
    const T *pz = p + z * N;
    double sZ = 0.0, mD = -INFINITY, sP = 0.0, mP = -INFINITY;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const T G = Gz[x], hb = Hbz[x];
        if (mode == MODE_ITER) {
            const T Dv = -hb - G;
            reinterpret_cast<T *>(Dout)[z * N + x] = Dv;
            sZ += (double)(pz[x] * exp2_t<T>(Dv));
            mD = fmax(mD, (double)Dv);
        } else if (mode == MODE_DIV) {
            const double Dv = (double)(-hb - G) + I[I_SUMP];
            reinterpret_cast<double *>(Dout)[z * N + x] = Dv;
            mD = fmax(mD, Dv);
        } else if (mode == MODE_DUAL) {
            const double Dv = (double)(-hb - G) + I[I_NEGH];
            reinterpret_cast<double *>(Dout)[z * N + x] = Dv;
            mD = fmax(mD, Dv);
        } else if (mode == MODE_DUAL_D) {
            const double Dv = reinterpret_cast<const double *>(Dout)[z * N + x];
            const double pi = exp2((Dv - I[I_DUAL_MAXD]) / I[I_DUAL_TAU]) / I[I_DUAL_S];
            sZ += pi * (-hb2[z * N + x] - (double)G);
        } else {  // MODE_CERT: the certified value with its rounding margin
            const double Gd = (double)G, Hd = (double)hb;
            const double Dv = -Hd - Gd;
            const double m =
                __dadd_ru(__dmul_ru(eH_scale, fabs(Gd)), __dadd_ru(__dmul_ru(1.01 * u, fabs(Hd) + fabs(Gd)), I[I_EH]));
            reinterpret_cast<double *>(Dout)[z * N + x] = Dv;
            const double pv = (double)pz[x];
            sZ += pv * exp2(Dv);
            sP += pv;
            mD = fmax(mD, __dadd_ru(Dv, m));
            mP = fmax(mP, Dv);
        }
    }
    double v[4] = {sZ, mD, sP, mP};
    for (int j = 0; j < 4; j++) {
        const bool isMax = (j & 1) != 0;
        double t = v[j];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, t, o);
            t = isMax ? fmax(t, w) : t + w;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = isMax ? -INFINITY : 0.0;
            for (int w = 0; w < ST_THREADS / 32; w++) r = isMax ? fmax(r, red[w]) : r + red[w];
            v[j] = r;
        }
    }
    if (threadIdx.x == 0) {
        double *pp = part + ((size_t)z * 2 + 1) * maxblk * 4 + blockIdx.x * 4;
        if (mode == MODE_ITER) {
            pp[0] = v[0];
            pp[1] = v[1];
            pp[2] = 0.0;
            pp[3] = -INFINITY;
        } else {
            pp[0] = v[0];
            pp[1] = v[1];
            pp[2] = v[2];
            pp[3] = v[3];
        }
    }
}

int level_grid(size_t M) { return (int)std::min<size_t>((M + ST_THREADS - 1) / ST_THREADS, (size_t)148 * 32); }

}  // namespace

template <typename T>
bdc_status stream_forward(bdc_engine *e, PrecBuf<T> &b, const T *p_src, int apply_update, int mode) {
    const int n = e->n, nd = e->nd;
    const size_t M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    T *A = b.Tm, *B = b.Gb;  // two code-indexed [nd][2^(n+1)] buffers
    k_stream_init_fwd<T><<<dim3(b.s.nblk_cols, nd), ST_THREADS, 0, e->stream>>>(
        n, const_cast<T *>(p_src), b.D, A, b.part, maxblk, e->inst, apply_update);
    e->launches++;
    const dim3 g(level_grid(M), nd);
    for (int i = 0; i < n; i++) {
        k_stream_fwd<T><<<g, ST_THREADS, 0, e->stream>>>(n, i, A, B, e->inst);
        e->launches++;
        std::swap(A, B);
    }
    k_stream_q<T><<<g, ST_THREADS, 0, e->stream>>>(n, A, b.q, b.L, e->bk + (size_t)4 * nd * (n + 1),
                                                   e->opt.q_floor, mode, e->inst);
    e->launches++;
    stage_mark(e, "stream_fwd");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template <typename T>
bdc_status stream_adjoint(bdc_engine *e, PrecBuf<T> &b, const T *Lsrc, const T *omega, T *Dout, int mode) {
    const int n = e->n, nd = e->nd;
    const size_t M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    T *A = b.Tm, *B = b.Gb;
    const dim3 g(level_grid(M), nd);
    k_stream_init_adj<T><<<g, ST_THREADS, 0, e->stream>>>(n, Lsrc, omega, A, e->inst);
    e->launches++;
    for (int i = n - 1; i >= 0; i--) {
        k_stream_adj<T><<<g, ST_THREADS, 0, e->stream>>>(n, i, A, B, e->inst);
        e->launches++;
        std::swap(A, B);
    }
    const double u = 1.1102230246251565e-16, mm = n + 8;
    const double eH_scale = 1.01 * (mm * u / (1.0 - mm * u)) + 1.01 * u;  // gamma_{n+8} * 1.01 + 1.01 u
    const T *p = (mode == MODE_CERT) ? reinterpret_cast<const T *>(e->pcert) : b.p;
    k_stream_epi<T><<<dim3(b.s.nblk_cols, nd), ST_THREADS, 0, e->stream>>>(
        n, A, b.Hb, p, Dout, e->pcert, b.part, maxblk, e->inst, mode, eH_scale, u);
    e->launches++;
    stage_mark(e, "stream_adj");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template bdc_status stream_forward<float>(bdc_engine *, PrecBuf<float> &, const float *, int, int);
template bdc_status stream_forward<double>(bdc_engine *, PrecBuf<double> &, const double *, int, int);
template bdc_status stream_adjoint<float>(bdc_engine *, PrecBuf<float> &, const float *, const float *, float *, int);
template bdc_status stream_adjoint<double>(bdc_engine *, PrecBuf<double> &, const double *, const double *, double *,
                                           int);
