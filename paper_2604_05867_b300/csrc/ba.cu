// Blahut-Arimoto glue (Sec. 2.3): per-d entropy term from the d-free
// precompute, the end-of-iteration reduction (bounds, stopping test, BA
// normalisation), orbit symmetrisation of D (Appendix A), the deferred
// p update, and the literal path's update on orbit representatives.
//
// Decomposition used by the sweep path (b_k = C(n,k) d^(n-k) (1-d)^k, the
// probability that exactly k symbols survive; P_{n,k} the exact channel):
//   W(y|x) = b_k P_{n,k}(y|x),  q(y) = b_k q_k(y)
//   D_x = sum_k b_k D(P_{n,k}(.|x) || q_k)
//       = -Hb(x) - sum_y (b_k / C(n,k)) Count(y,x) log2 q_k(y) + log2 sum_x p(x)
//   Hb(x) = sum_k b_k H_k(x),  H_k(x) = log2 C(n,k) - S_k(x) / C(n,k),
//   S_k(x) = sum_{|y|=k} Count log2 Count   (d-free, computed once per n).
#include "bdc_internal.cuh"

#include <algorithm>

namespace {

__device__ __forceinline__ int64_t find_rep(const uint32_t *reps, int64_t R, uint32_t r) {
    int64_t lo = 0, hi = R - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (reps[mid] < r) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void k_build_Hb(int n, int nd, const uint32_t *reps, int64_t R, const double *Sk, const double *bk,
                           const double *lc, const double *ic, T *Hb) {
    const size_t N = (size_t)1 << n;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        uint32_t r = orbit_rep_dev((uint32_t)x, n, nullptr);
        int64_t idx = find_rep(reps, R, r);
        const double *S = Sk + idx * (n + 1);
        for (int z = 0; z < nd; z++) {
            const double *b = bk + z * (n + 1);
            double h = 0.0;
            for (int k = 0; k <= n; k++) h += b[k] * (lc[k] - S[k] * ic[k]);
            Hb[z * N + x] = (T)h;
        }
    }
}

// one block per instance; partials reduced in a fixed order (deterministic)
__global__ void k_finalize_iter(int nd, const double *part, int maxblk, int nblk0, int nblk1, double *inst,
                                double *hist, int stepped) {
    __shared__ double red[FIN_THREADS / 32];
    const int z = blockIdx.x;
    if (inst[z * INST_STRIDE + I_ACTIVE] == 0.0) return;
    finalize_instance<FIN_THREADS>(z, part, maxblk, nblk0, nblk1, inst, hist, stepped, red);
}

// sum of slot-0 partials -> inst[I_SUMP] = log2(sum)
// (add_negh: q is a full output marginal, so the length entropy -h(b) does
// not cancel and joins the constant)
__global__ void k_finalize_sum(int nd, const double *part, int maxblk, int nblk, double *inst, int add_negh) {
    __shared__ double red[FIN_THREADS / 32];
    const int z = blockIdx.x;
    const double *p0 = part + ((size_t)z * 2 + 0) * maxblk * 4;
    double s = fin_sum(p0, 4, nblk, red);
    if (threadIdx.x == 0)
        inst[z * INST_STRIDE + I_SUMP] = log2(s) + (add_negh ? inst[z * INST_STRIDE + I_NEGH] : 0.0);
}

// orbit mean of D (Appendix A symmetry).  x = (h | mid | l) with hb-bit h and
// l; the orbit of x only touches the tiles of mid, cpl mid, rev mid and
// cpl rev mid, so one CTA per representative mid loads those tiles, and the
// thread owning the orbit representative writes one canonical mean to all
// members (bit-identical across the orbit).
// n2h > 0: complement half mode, only inputs whose bit (n2h-1) is 0 are
// stored and written; the others are read as their complements
template <typename T>
__global__ void k_symmetrize(int n, T *D, const double *inst, int n2h, int force) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    const int z = blockIdx.y;
    if (!force && inst[z * INST_STRIDE + I_SYMNEED] == 0.0) return;
    const int hb = min(5, n / 2), nm = n - 2 * hb;
    const uint32_t H = 1u << hb, TS = H * H;
    const uint32_t mid = blockIdx.x;
    if (orbit_rep_dev(mid, nm, nullptr) != mid) return;
    const uint32_t mm = nm ? ((1u << nm) - 1u) : 0u;
    uint32_t cand[4] = {mid, mid ^ mm, rev_bits(mid, nm), rev_bits(mid, nm) ^ mm};
    uint32_t mids[4];
    int nt = 0;
    for (int t = 0; t < 4; t++) {
        bool seen = false;
        for (int s = 0; s < nt; s++) seen |= (mids[s] == cand[t]);
        if (!seen) mids[nt++] = cand[t];
    }
    T *Dz = D + ((size_t)z << n);
    // tile rows padded to H+1 elements: the reversed reads hit distinct banks
    const uint32_t HP = H + 1u, TSP = H * HP, lg = 2 * hb;
    for (uint32_t e = threadIdx.x; e < nt * TS; e += blockDim.x) {
        uint32_t t = e >> lg, r = e & (TS - 1u);
        uint32_t h = r >> hb, l = r & (H - 1u);
        size_t x = ((size_t)h << (n - hb)) | ((size_t)mids[t] << hb) | l;
        if (n2h && ((x >> (n2h - 1)) & 1u)) x ^= (size_t)((1u << n) - 1u);
        tile[t * TSP + h * HP + l] = Dz[x];
    }
    __syncthreads();
    // every element: the mean over its orbit, summed in the order of the
    // orbit representative's members, so all members get the same bits
    const uint32_t full = (1u << n) - 1u;
    for (uint32_t e = threadIdx.x; e < nt * TS; e += blockDim.x) {
        uint32_t t = e >> lg, r = e & (TS - 1u);
        uint32_t h = r >> hb, l = r & (H - 1u);
        uint32_t x = (h << (n - hb)) | (mids[t] << hb) | l;
        uint32_t rp = orbit_rep_dev(x, n, nullptr);
        uint32_t rr = rev_bits(rp, n);
        uint32_t mem[4] = {rp, rp ^ full, rr, rr ^ full};
        T v[4];
        for (int s = 0; s < 4; s++) {
            uint32_t y = mem[s];
            uint32_t ym = (y >> hb) & mm;
            int ti = 0;
            for (int q = 0; q < nt; q++)
                if (mids[q] == ym) ti = q;
            v[s] = tile[ti * TSP + (y >> (n - hb)) * HP + (y & (H - 1u))];
        }
        if (n2h && ((x >> (n2h - 1)) & 1u)) continue;
        Dz[x] = ((v[0] + v[1]) + (v[2] + v[3])) * (T)0.25;
    }
}

// complement half mode -> full arrays: a[x] = a[cpl x] where bit (n2-1) of x is 1
template <typename T>
__global__ void k_mirror_half(int n, int n2, int nd, T *a) {
    const size_t N = (size_t)1 << n;
    const uint32_t full = (1u << n) - 1u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * nd; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(i & (N - 1));
        if ((x >> (n2 - 1)) & 1u) a[i] = a[(i & ~(N - 1)) | (x ^ full)];
    }
}

template <typename T>
__global__ void k_apply_pending(int n, int nd, T *p, const T *D, double *inst) {
    const size_t N = (size_t)1 << n;
    for (int z = 0; z < nd; z++) {
        const double *I = inst + z * INST_STRIDE;
        if (I[I_PENDING] == 0.0) continue;
        T sh = (T)I[I_SHIFT];
        for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x)
            p[z * N + x] = p[z * N + x] * exp2_t<T>(D[z * N + x] - sh);
    }
}

__global__ void k_clear_pending(int nd, double *inst) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < nd) inst[z * INST_STRIDE + I_PENDING] = 0.0;
}

// a stepped sequence starts from shift 0, so that it depends on p alone (a
// resumed checkpoint continues bit for bit)
__global__ void k_reset_shift(int nd, double *inst) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < nd) inst[z * INST_STRIDE + I_SHIFT] = 0.0;
}

__global__ void k_clear_symneed(int nd, double *inst) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < nd) inst[z * INST_STRIDE + I_SYMNEED] = 0.0;
}

// literal path, on representatives: apply the pending update to every orbit
// member, and the orbit-weighted partial sums of p (slot 0)
__global__ void k_literal_update(int n, int64_t R, const uint32_t *reps, const uint8_t *osize, double *p,
                                 const double *Dr, double *part, int maxblk, double *inst) {
    __shared__ double red[32];
    const int z = blockIdx.y;
    double *I = inst + z * INST_STRIDE;
    if (I[I_ACTIVE] == 0.0) return;
    const bool upd = I[I_PENDING] != 0.0;
    const double sh = I[I_SHIFT];
    double *pz = p + ((size_t)z << n);
    const double *Dz = Dr + (size_t)z * R;
    const uint32_t full = (1u << n) - 1u;
    double s = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = reps[r];
        double v = pz[x];
        if (upd) {
            v = v * exp2(Dz[r] - sh);
            uint32_t rx = rev_bits(x, n);
            pz[x] = v;
            pz[x ^ full] = v;
            pz[rx] = v;
            pz[rx ^ full] = v;
        }
        s += v * (double)osize[r];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[((size_t)z * 2 + 0) * maxblk * 4 + blockIdx.x * 4] = t;
    }
}

// literal path: Z = sum_r |O_r| p_r 2^{D_r}, max D (slot 1)
__global__ void k_literal_reduce(int n, int64_t R, const uint32_t *reps, const uint8_t *osize, const double *p,
                                 const double *Dr, double *part, int maxblk, const double *inst) {
    __shared__ double red[32], redm[32];
    const int z = blockIdx.y;
    if (inst[z * INST_STRIDE + I_ACTIVE] == 0.0) return;
    const double *pz = p + ((size_t)z << n);
    const double *Dz = Dr + (size_t)z * R;
    double s = 0.0, m = -INFINITY;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        double D = Dz[r];
        s += (double)osize[r] * pz[reps[r]] * exp2(D);
        m = fmax(m, D);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        redm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, tm = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t += red[w];
            tm = fmax(tm, redm[w]);
        }
        double *pp = part + ((size_t)z * 2 + 1) * maxblk * 4 + blockIdx.x * 4;
        pp[0] = t;
        pp[1] = tm;
    }
}

// expand literal D on reps to every input x (for bdc_divergence / get)
__global__ void k_expand_reps(int n, int nd, int64_t R, const uint32_t *reps, const double *Dr, double *out) {
    const uint32_t full = (1u << n) - 1u;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = reps[r], rx = rev_bits(x, n);
        for (int z = 0; z < nd; z++) {
            double v = Dr[(size_t)z * R + r];
            double *o = out + ((size_t)z << n);
            o[x] = v;
            o[x ^ full] = v;
            o[rx] = v;
            o[rx ^ full] = v;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(size_t n, int threads, int cap = 148 * 32) {
    size_t g = (n + threads - 1) / threads;
    return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)cap));
}

template <typename T>
bdc_status launch_build_Hb(bdc_engine *e, PrecBuf<T> &b) {
    const int n = e->n;
    const double *lc = e->bk + (size_t)5 * e->nd * (n + 1);
    const double *ic = e->bk + (size_t)4 * e->nd * (n + 1);
    k_build_Hb<T><<<grid_for((size_t)1 << n, 256), 256, 0, e->stream>>>(n, e->nd, e->reps, e->R, e->Sk, e->bk, lc,
                                                                         ic, b.Hb); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

int part_maxblk(const bdc_engine *e);

// sum_k w_k H_k(x) for per-instance weights w [nd][n+1] (FP64)
bdc_status launch_build_Hb_w(bdc_engine *e, const double *w, double *out) {
    const int n = e->n;
    const double *lc = e->bk + (size_t)5 * e->nd * (n + 1);
    const double *ic = e->bk + (size_t)4 * e->nd * (n + 1);
    k_build_Hb<double><<<grid_for((size_t)1 << n, 256), 256, 0, e->stream>>>(n, e->nd, e->reps, e->R, e->Sk, w, lc,
                                                                              ic, out);
    e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template <typename T>
bdc_status launch_finalize(bdc_engine *e, PrecBuf<T> &b, int mode, int add_negh, int nblk, int stepped) {
    int maxblk = part_maxblk(e);
    if (nblk <= 0) nblk = b.s.nblk_cols;
    if (mode == MODE_ITER) {
        k_finalize_iter<<<e->nd, FIN_THREADS, 0, e->stream>>>(e->nd, b.part, maxblk, nblk, nblk, e->inst, e->hist,
                                                              stepped); e->launches++; stage_mark(e, "finalize");
    } else {
        k_finalize_sum<<<e->nd, FIN_THREADS, 0, e->stream>>>(e->nd, b.part, maxblk, b.s.nblk_cols, e->inst,
                                                             add_negh); e->launches++;
    }
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_finalize_literal(bdc_engine *e, int nblk0, int nblk1) {
    k_finalize_iter<<<e->nd, FIN_THREADS, 0, e->stream>>>(e->nd, e->f64.part, part_maxblk(e), nblk0, nblk1, e->inst,
                                                          e->hist, 0); e->launches++; stage_mark(e, "finalize");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template <typename T>
bdc_status launch_mirror_half(bdc_engine *e, T *a, int n2) {
    k_mirror_half<T><<<grid_for((size_t)e->nd << e->n, 256), 256, 0, e->stream>>>(e->n, n2, e->nd, a); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template <typename T>
bdc_status launch_symmetrize(bdc_engine *e, T *D, int n2h, bool force) {
    const int n = e->n;
    const int hb = std::min(5, n / 2), nm = n - 2 * hb;
    size_t smem = (size_t)4 * ((size_t)1 << hb) * (((size_t)1 << hb) + 1) * sizeof(T);
    dim3 g(1u << nm, e->nd);
    k_symmetrize<T><<<g, 256, smem, e->stream>>>(n, D, e->inst, n2h, force ? 1 : 0); e->launches++;
    if (!force) {
        k_clear_symneed<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst); e->launches++;
    }
    stage_mark(e, "symmetrize");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template <typename T>
bdc_status launch_apply_pending(bdc_engine *e, PrecBuf<T> &b) {
    k_apply_pending<T><<<grid_for((size_t)1 << e->n, 256), 256, 0, e->stream>>>(e->n, e->nd, b.p, b.D, e->inst); e->launches++;
    k_clear_pending<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_reset_shift(bdc_engine *e) {
    k_reset_shift<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_clear_symneed(bdc_engine *e) {
    k_clear_symneed<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_clear_pending(bdc_engine *e) {
    k_clear_pending<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

int literal_grid(const bdc_engine *e) { return std::min<int>(part_maxblk(e), grid_for((size_t)e->R, 256, 1024)); }

bdc_status launch_literal_update(bdc_engine *e) {
    dim3 g(literal_grid(e), e->nd);
    k_literal_update<<<g, 256, 0, e->stream>>>(e->n, e->R, e->reps, e->osize, e->lit_p, e->lit_D, e->f64.part,
                                              part_maxblk(e), e->inst); e->launches++; stage_mark(e, "literal_update");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_literal_reduce(bdc_engine *e) {
    dim3 g(literal_grid(e), e->nd);
    k_literal_reduce<<<g, 256, 0, e->stream>>>(e->n, e->R, e->reps, e->osize, e->lit_p, e->lit_D, e->f64.part,
                                              part_maxblk(e), e->inst); e->launches++; stage_mark(e, "literal_reduce");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_expand_reps(bdc_engine *e, const double *Dr, double *out) {
    k_expand_reps<<<grid_for((size_t)e->R, 256), 256, 0, e->stream>>>(e->n, e->nd, e->R, e->reps, Dr, out); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template bdc_status launch_build_Hb<float>(bdc_engine *, PrecBuf<float> &);
template bdc_status launch_build_Hb<double>(bdc_engine *, PrecBuf<double> &);
template bdc_status launch_finalize<float>(bdc_engine *, PrecBuf<float> &, int, int, int, int);
template bdc_status launch_finalize<double>(bdc_engine *, PrecBuf<double> &, int, int, int, int);
template bdc_status launch_symmetrize<float>(bdc_engine *, float *, int, bool);
template bdc_status launch_symmetrize<double>(bdc_engine *, double *, int, bool);
template bdc_status launch_mirror_half<float>(bdc_engine *, float *, int);
template bdc_status launch_mirror_half<double>(bdc_engine *, double *, int);
template bdc_status launch_apply_pending<float>(bdc_engine *, PrecBuf<float> &);
template bdc_status launch_apply_pending<double>(bdc_engine *, PrecBuf<double> &);
