// C ABI of libbdc: engine lifecycle, workspace layout, the d-free precompute,
// the iteration driver (CUDA-graph replay), divergence, certification and
// state access.  See include/bdc.h for the contract of every entry point.
#include "bdc_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

static thread_local std::string g_err;
void bdc_set_error(const std::string &m) { g_err = m; }
extern "C" const char *bdc_last_error(void) { return g_err.c_str(); }

#define BDC_FAIL(code, msg)        \
    do {                           \
        bdc_set_error(msg);        \
        return code;               \
    } while (0)

double binom_d(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    long double r = 1.0L;
    for (int i = 1; i <= k; i++) r = r * (long double)(n - k + i) / (long double)i;
    return (double)floorl(r + 0.5L);
}

int part_maxblk(const bdc_engine *e) {
    return std::max(1024, std::max(e->f32.s.nblk_cols, e->f64.s.nblk_cols));
}

static inline double gamma_u(double m) {
    const double u = 1.1102230246251565e-16;
    return m * u / (1.0 - m * u);
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
namespace {

__global__ void k_activate(int nd, double *inst, double tol) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nd) return;
    double *I = inst + z * INST_STRIDE;
    I[I_ACTIVE] = 1.0;
    I[I_TOL] = tol;
    I[I_ITERS] = 0.0;
    I[I_STATUS] = 0.0;
}

template <typename T>
__global__ void k_fill(T *a, size_t count, T v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        a[i] = v;
}

template <typename S, typename D>
__global__ void k_convert(const S *src, D *dst, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

// per-instance sums over [nd][count] into part slot 0 (block order fixed)
// mode 0: plain sum of every entry; 1: code array (slot 0 skipped);
// 2: code array, sum of wk[z][k] * min(v, 1) (wk may be NULL: weight 1)
template <typename T>
__global__ void k_sum_rows(const T *a, size_t count, double *part, int maxblk, int mode, const double *wk, int n) {
    __shared__ double red[32];
    const int z = blockIdx.y;
    const T *az = a + z * count;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        if (mode > 0 && i == 0) continue;
        double v = (double)az[i];
        if (mode == 2) {
            v = fmin(v, 1.0);
            if (wk) v = v * wk[z * (n + 1) + (bitlen32((uint32_t)i) - 1)];
        }
        s += v;
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

// certify input: p~ = (1 - eps) p / sum p + eps 2^-n
template <typename T>
__global__ void k_make_pcert(int n, int nd, const T *p, const double *inst, double eps, double *out) {
    const size_t N = (size_t)1 << n;
    for (int z = 0; z < nd; z++) {
        double inv = exp2(-inst[z * INST_STRIDE + I_SUMP]);
        double u = eps * exp2(-(double)n);
        for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x)
            out[z * N + x] = (1.0 - eps) * ((double)p[z * N + x] * inv) + u;
    }
}

template <typename T>
__global__ void k_log2_codes_nd(const T *q, T *L, size_t per, int nd, int min1) {
    size_t total = per * nd;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        if (i % per == 0) { L[i] = (T)0; continue; }
        T v = q[i];
        if (min1) v = v < (T)1 ? v : (T)1;
        L[i] = log2_t<T>(v);
    }
}

// a caller-given output distribution must be finite and positive at every
// code: record BDC_ENONFINITE (NaN or Inf) or BDC_EINVAL (<= 0) per instance
__global__ void k_check_given_q(const double *q, size_t M, double *inst) {
    const int z = blockIdx.y;
    const double *qz = q + z * M;
    int bad = 0;
    for (size_t c = 1 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (size_t)gridDim.x * blockDim.x) {
        const double v = qz[c];
        if (!isfinite(v)) bad |= 2;
        else if (!(v > 0.0)) bad |= 1;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) {
        double *st = inst + z * INST_STRIDE + I_STATUS;
        // (where both kinds occur, either status may be the one recorded)
        if (bad & 2) *st = (double)BDC_ENONFINITE;
        else if (*st == 0.0) *st = (double)BDC_EINVAL;
    }
}

// checks of an input distribution given by the caller (instance z = blockIdx.y):
// flags[z] |= 1 if an entry is negative or not finite, 2 if p(x) != p(cpl x)
// for some x, 4 if p(x) != p(rev x); block sums of p into part slot 0
__global__ void k_check_p(int n, const double *p, uint32_t *flags, double *part, int maxblk) {
    __shared__ double red[32];
    const int z = blockIdx.y;
    const size_t N = (size_t)1 << n, full = N - 1;
    const double *pz = p + z * N;
    uint32_t f = 0;
    double s = 0.0;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x) {
        const double v = pz[x];
        if (!(v >= 0.0) || !isfinite(v)) f |= 1u;
        if (v != pz[x ^ full]) f |= 2u;
        if (v != pz[rev_bits((uint32_t)x, n)]) f |= 4u;
        s += v;
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags + z, f);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[((size_t)z * 2 + 0) * maxblk * 4 + blockIdx.x * 4] = t;
    }
}

// flags[z] |= 1 where some p(x) differs from p(cpl x) (bitwise)
__global__ void k_check_cpl(int n, const double *p, uint32_t *flags) {
    const int z = blockIdx.y;
    const size_t N = (size_t)1 << n, full = N - 1;
    const double *pz = p + z * N;
    uint32_t f = 0;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N / 2; x += (size_t)gridDim.x * blockDim.x)
        if (pz[x] != pz[x ^ full]) f = 1u;
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags + z, f);
}

// p <- p / sum p per instance, the sum taken from the nb block partials of
// k_check_p (in block order: every CTA forms the same value)
__global__ void k_normalize_p(int n, double *p, const double *part, int maxblk, int nb) {
    __shared__ double red[FIN_THREADS / 32];
    __shared__ double tot_s;
    const int z = blockIdx.y;
    const double tot = fin_sum(part + ((size_t)z * 2 + 0) * maxblk * 4, 4, nb, red);
    if (threadIdx.x == 0) tot_s = tot;
    __syncthreads();
    const double t = tot_s;
    const size_t N = (size_t)1 << n;
    double *pz = p + z * N;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (size_t)gridDim.x * blockDim.x)
        pz[x] = pz[x] / t;
}

// certified upper bound: U = max_x up(D'_x + m_x) + up(log2 sum q~ + e_Lambda)
__global__ void k_finalize_cert(int nd, const double *part, int maxblk, int nb0, int nb1, double Kterms,
                                int have_lower, double *inst) {
    __shared__ double red[FIN_THREADS / 32];
    const int z = blockIdx.x;
    const double u = 1.1102230246251565e-16;
    const double *p0 = part + ((size_t)z * 2 + 0) * maxblk * 4;
    const double *p1 = part + ((size_t)z * 2 + 1) * maxblk * 4;
    double sq = fin_sum(p0, 4, nb0, red);
    double S1 = fin_sum(p1, 4, nb1, red);
    double mUp = fin_max(p1 + 1, 4, nb1, red);
    double Sp = fin_sum(p1 + 2, 4, nb1, red);
    double mPl = fin_max(p1 + 3, 4, nb1, red);
    if (threadIdx.x != 0) return;
    double *I = inst + z * INST_STRIDE;
    double Lam = log2(sq);
    double g = (Kterms + 3.0) * u / (1.0 - (Kterms + 3.0) * u);
    double eL = __dadd_ru(__dmul_ru(1.01 * g, 1.4426950408889634), __dmul_ru(2.02 * u, fabs(Lam)));
    if (!have_lower) {
        // full output marginal: the length entropy -h(b) joins the constant
        double ng = I[I_NEGH];
        Lam = Lam + ng;
        eL = __dadd_ru(eL, __dmul_ru(4.0 * u, fabs(ng) + fabs(Lam)));
    }
    double U = __dadd_ru(mUp, __dadd_ru(Lam, eL));
    I[I_CERT_U] = U;
    I[I_CERT_M] = U - (mPl + Lam);
    I[I_LOG2SQ] = Lam;
    I[I_LOG2SQ_ERR] = eL;
    I[I_CERT_LO] = have_lower ? (log2(S1 / Sp) + Lam) : NAN;
    if (!isfinite(U) && I[I_STATUS] == 0.0) I[I_STATUS] = (double)BDC_ENONFINITE;
}

int grid_for(size_t n, int threads, int cap = 148 * 32) {
    size_t g = (n + threads - 1) / threads;
    return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)cap));
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

template <typename T>
void carve_prec(Carver &c, PrecBuf<T> &b, int n, int nd, int maxblk) {
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;
    b.p = c.take<T>(nd * N);
    b.D = c.take<T>(nd * N);
    b.Hb = c.take<T>(nd * N);
    b.q = c.take<T>(nd * M);
    b.L = c.take<T>(nd * M);
    b.aux = c.take<T>(nd * M);
    b.pd = c.take<T>(nd * N);
    b.omega = c.take<T>((size_t)nd * (n + 1));
    b.omega2 = c.take<T>((size_t)nd * (n + 1));
    b.part = c.take<double>((size_t)nd * 2 * maxblk * 4);
    if (b.s.n2 != 0 || n >= 15) {
        // sized for every split the autotuner may choose (n2 >= 8, so n1 <= n - 8);
        // the streaming schedule (n2 < 0) ping-pongs between Tm and Gb
        int n1max = std::max(b.s.n2 > 0 ? b.s.n1 : 0, n - 8);
        b.F1 = c.take<T>(nd * N);
        b.Tm = c.take<T>(nd * M);
        b.Ts = c.take<T>((size_t)nd * 32 * ((size_t)2 << n1max));
        b.Gb = c.take<T>(nd * M);
    } else {
        b.F1 = b.Tm = b.Ts = b.Gb = nullptr;
    }
}

size_t carve(bdc_engine *e, char *base) {
    Carver c{base, 0};
    const int n = e->n, nd = e->nd;
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    e->reps = c.take<uint32_t>(e->R);
    e->osize = c.take<uint8_t>(e->R);
    e->Nk = c.take<uint32_t>((size_t)e->R * (n + 1));
    e->Sk = c.take<double>((size_t)e->R * (n + 1));
    e->oreps = c.take<uint32_t>(e->Rout);
    e->ocls = c.take<int32_t>(M);
    e->counter = c.take<uint32_t>(64 + 2 * (size_t)nd);
    e->pflags = c.take<uint32_t>((size_t)nd);
    e->scan_tmp = c.take<uint32_t>(M / 2048 + 16);
    e->bk = c.take<double>((size_t)6 * nd * (n + 1));
    e->tab_clog = c.take<double>(8192);
    e->tab_fix = c.take<longlong2>(65536);
    e->inst = c.take<double>((size_t)nd * INST_STRIDE);
    e->hist = c.take<double>((size_t)nd * 2 * BDC_HIST);
    e->pcert = c.take<double>(nd * N);
    e->marg = c.take<double>(nd * N);
    e->dual_w = c.take<double>((size_t)nd * (n + 1));
    if (e->opt.enable_literal) {
        e->lit_part = c.take<double>(literal_part_bytes(n, nd) / sizeof(double) + 1);
        e->lit_q = c.take<double>(nd * M);
        e->lit_L = c.take<double>(nd * M);
        e->lit_p = c.take<double>(nd * N);
        e->lit_D = c.take<double>((size_t)nd * e->R);
    }
    carve_prec(c, e->f32, n, nd, maxblk);
    carve_prec(c, e->f64, n, nd, maxblk);
    return c.off + 256;
}

}  // namespace

// ---------------------------------------------------------------------------
// lifecycle
// ---------------------------------------------------------------------------
extern "C" void bdc_default_options(bdc_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->symmetrize = 1;
    o->use_graph = 1;
    o->chunk = 8;
    o->q_floor = 1e-30;
    o->certify_mix = 9.313225746154785e-10;  // 2^-30
    o->enable_literal = 1;
    o->use_half = 1;
    o->use_regsteps = 15;
    o->fuse_update = 1;
    o->use_tma = 0;
}

static bdc_engine *new_engine(int n, int nd, const bdc_options *opt);

extern "C" bdc_status bdc_create(int n, const double *d, int nd, const bdc_options *opt, bdc_engine **out) {
    if (!out) BDC_FAIL(BDC_EINVAL, "bdc_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n > BDC_MAXN) BDC_FAIL(BDC_EINVAL, "bdc_create: n must be in [1, 28]");
    if (!d || nd < 1 || nd > 4096) BDC_FAIL(BDC_EINVAL, "bdc_create: need 1 <= nd <= 4096 values of d");
    for (int i = 0; i < nd; i++)
        if (!(d[i] >= 0.0 && d[i] <= 1.0)) BDC_FAIL(BDC_EINVAL, "bdc_create: every d must lie in [0, 1]");
    bdc_engine *e = new_engine(n, nd, opt);
    e->d.assign(d, d + nd);
    *out = e;
    return BDC_OK;
}

extern "C" bdc_status bdc_create_lengths(int n, const double *b, int nb, const bdc_options *opt, bdc_engine **out) {
    if (!out) BDC_FAIL(BDC_EINVAL, "bdc_create_lengths: out is NULL");
    *out = nullptr;
    if (n < 1 || n > BDC_MAXN) BDC_FAIL(BDC_EINVAL, "bdc_create_lengths: n must be in [1, 28]");
    if (!b || nb < 1 || nb > 4096) BDC_FAIL(BDC_EINVAL, "bdc_create_lengths: need 1 <= nb <= 4096 length distributions");
    std::vector<double> bl((size_t)nb * (n + 1));
    for (int z = 0; z < nb; z++) {
        long double s = 0.0L;
        for (int k = 0; k <= n; k++) {
            double v = b[(size_t)z * (n + 1) + k];
            if (!(v >= 0.0) || !std::isfinite(v))
                BDC_FAIL(BDC_EINVAL, "bdc_create_lengths: every b_k must be finite and non-negative");
            s += v;
        }
        if (!(s > 0.0L)) BDC_FAIL(BDC_EINVAL, "bdc_create_lengths: every length distribution needs a positive sum");
        for (int k = 0; k <= n; k++) bl[(size_t)z * (n + 1) + k] = (double)(b[(size_t)z * (n + 1) + k] / s);
    }
    bdc_engine *e = new_engine(n, nb, opt);
    e->d.assign(nb, std::nan(""));
    e->blen = bl;
    *out = e;
    return BDC_OK;
}

static bdc_engine *new_engine(int n, int nd, const bdc_options *opt) {
    bdc_engine *e = new bdc_engine();
    e->n = n;
    e->nd = nd;
    if (opt) e->opt = *opt;
    else bdc_default_options(&e->opt);
    if (e->opt.chunk < 1) e->opt.chunk = 1;
    e->R = num_reps_host(n);
    e->Rout = 0;
    for (int k = 0; k <= n; k++) e->Rout += num_reps_host(k);
    e->f32.s = make_sched(n, 4, e->opt.sched_n2_fp32, e->opt.sched_w_fp32);
    e->f64.s = make_sched(n, 8, e->opt.sched_n2_fp64, e->opt.sched_w_fp64);
    e->ws_bytes = carve(e, nullptr);
    return e;
}

extern "C" size_t bdc_workspace_bytes(const bdc_engine *e) { return e ? e->ws_bytes : 0; }

extern "C" void bdc_destroy(bdc_engine *e) {
    if (!e) return;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            if (e->graph[a][b]) cudaGraphExecDestroy(e->graph[a][b]);
            if (e->graph1[a][b]) cudaGraphExecDestroy(e->graph1[a][b]);
        }
    if (e->prof_created)
        for (int i = 0; i < 32; i++) cudaEventDestroy(e->prof_ev[i]);
    delete e;
}

static bdc_status sync_check(bdc_engine *e, const char *what) {
    cudaError_t err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        bdc_set_error(std::string(what) + ": " + cudaGetErrorString(err));
        return BDC_ECUDA;
    }
    return BDC_OK;
}

static bdc_status read_inst(bdc_engine *e, std::vector<double> &h) {
    h.resize((size_t)e->nd * INST_STRIDE);
    BDC_CUDA_TRY(cudaMemcpyAsync(h.data(), e->inst, h.size() * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    return sync_check(e, "read instance state");
}

static bdc_status activate(bdc_engine *e, double tol) {
    k_activate<<<(e->nd + 63) / 64, 64, 0, e->stream>>>(e->nd, e->inst, tol); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

extern "C" bdc_status bdc_bind(bdc_engine *e, void *ws, size_t bytes, void *stream) {
    if (!e) BDC_FAIL(BDC_EINVAL, "bdc_bind: engine is NULL");
    if (!ws) BDC_FAIL(BDC_EINVAL, "bdc_bind: workspace is NULL");
    if (bytes < e->ws_bytes) BDC_FAIL(BDC_ENOMEM, "bdc_bind: workspace smaller than bdc_workspace_bytes()");
    if (((uintptr_t)ws) & 255) BDC_FAIL(BDC_EINVAL, "bdc_bind: workspace must be 256-byte aligned");
    e->ws = (char *)ws;
    e->stream = (cudaStream_t)stream;
    carve(e, e->ws);
    const int n = e->n, nd = e->nd;
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;

    // host tables: b_k, kw_k = d^(n-k)(1-d)^k, log2 kw, log2 b, 1/C(n,k), log2 C(n,k)
    std::vector<double> bk((size_t)6 * nd * (n + 1), 0.0);
    std::vector<double> rb((size_t)nd * (n + 1), 0.0), rw((size_t)nd * (n + 1), 0.0);
    std::vector<double> inst((size_t)nd * INST_STRIDE, 0.0);
    const bool lengths = !e->blen.empty();
    for (int z = 0; z < nd; z++) {
        long double d = lengths ? 0.5L : e->d[z], dm = 1.0L - d;
        double sum_blc = 0.0;
        long double negh = 0.0L, c0 = 0.0L;
        for (int k = 0; k <= n; k++) {
            // BDC_d: b_k = C(n,k) d^(n-k) (1-d)^k, one keep pattern weighs kw = b_k / C(n,k);
            // a length mixture (e.g. the exact channel BDC_{n,k}, Sec. 2.2): b_k given
            long double C = (long double)binom_d(n, k);
            long double kw = lengths ? (long double)e->blen[(size_t)z * (n + 1) + k] / C
                                     : powl(d, (long double)(n - k)) * powl(dm, (long double)k);
            long double b = lengths ? (long double)e->blen[(size_t)z * (n + 1) + k] : C * kw;
            size_t o = (size_t)z * (n + 1) + k, S = (size_t)nd * (n + 1);
            bk[o] = (double)b;
            bk[S + o] = (double)kw;
            bk[2 * S + o] = kw > 0 ? (double)log2l(kw) : 0.0;
            bk[3 * S + o] = b > 0 ? (double)log2l(b) : 0.0;
            bk[4 * S + o] = (double)(1.0L / C);
            bk[5 * S + o] = (double)log2l(C);
            sum_blc += (double)b * (double)log2l(C);
            if (b > 0) negh += b * log2l(b);
            // d-derivative weights: db_k/dd = rho_k b_k, rho_k = (n-k)/d - k/(1-d)
            if (!lengths && d > 0 && dm > 0) {
                long double rho = (long double)(n - k) / d - (long double)k / dm;
                rb[o] = (double)(rho * b);
                rw[o] = (double)(rho * kw);
                c0 += rho * b * (b > 0 ? log2l(b) : 0.0L);
            }
        }
        double *I = &inst[(size_t)z * INST_STRIDE];
        I[I_ACTIVE] = 1.0;
        I[I_TOL] = -1.0;
        // certified bound on |Hb^ - Hb|: S_k is an exact integer sum of terms
        // each within 2^-43 (long double table, |term| < 2^20, plus the 2^-62
        // fraction rounding) or 4u relative + 2^-62 (counts >= 65536, FP64) of
        // count*log2(count), converted with one rounding; with N_k <= C(n,k)
        // and S_k/C(n,k) <= log2 C(n,k): |H^_k - H_k| <= 2^-43 + 9u log2 C(n,k),
        // then the products and the (n+1)-term sum:
        // 1.05 (2^-43 + gamma_{n+14} sum_k b_k log2 C(n,k))
        I[I_EH] = 1.05 * (std::ldexp(1.0, -43) + gamma_u((double)n + 14) * sum_blc);
        I[I_NEGH] = (double)negh;
        I[I_DUAL_C0] = (double)c0;
    }
    std::vector<double> tab(8192, 0.0);
    for (int c = 1; c < 4096; c++) {
        tab[c] = (double)((long double)c * log2l((long double)c));
        tab[4096 + c] = (double)log2l((long double)c);
    }
    std::vector<longlong2> tabfix(65536);
    for (int c = 0; c < 65536; c++) {
        long double t = c < 2 ? 0.0L : (long double)c * log2l((long double)c);
        long double ip = floorl(t);
        unsigned long long f = (unsigned long long)llrintl((t - ip) * 4611686018427387904.0L);  // 2^62
        long long i = (long long)ip;
        if (f >= (1ull << 62)) { f -= (1ull << 62); i += 1; }
        tabfix[c].x = i;
        tabfix[c].y = (long long)f;
    }
    BDC_CUDA_TRY(cudaMemcpyAsync(e->bk, bk.data(), bk.size() * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(e->dual_w, rb.data(), rb.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(e->f64.omega2, rw.data(), rw.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(e->tab_clog, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(e->tab_fix, tabfix.data(), tabfix.size() * sizeof(longlong2),
                                 cudaMemcpyHostToDevice, e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(e->inst, inst.data(), inst.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 e->stream));
    BDC_CUDA_TRY(cudaMemsetAsync(e->counter, 0, (64 + 2 * (size_t)nd) * sizeof(uint32_t), e->stream));
    BDC_CUDA_TRY(cudaMemsetAsync(e->hist, 0, (size_t)nd * 2 * BDC_HIST * sizeof(double), e->stream));
    BDC_TRY(sync_check(e, "bdc_bind upload"));

    // d-free precompute: orbit reps, output classes, per-rep subsequence stats
    BDC_TRY(launch_reps(e));
    BDC_TRY(launch_output_classes(e));
    BDC_TRY(launch_subseq_stats(e));
    BDC_TRY(launch_build_Hb<float>(e, e->f32));
    BDC_TRY(launch_build_Hb<double>(e, e->f64));
    // adjoint weights omega_k = b_k / C(n,k) = d^(n-k)(1-d)^k
    const double *kw = e->bk + (size_t)nd * (n + 1);
    BDC_CUDA_TRY(cudaMemcpyAsync(e->f64.omega, kw, (size_t)nd * (n + 1) * sizeof(double), cudaMemcpyDeviceToDevice,
                                 e->stream));
    k_convert<double, float><<<1, 256, 0, e->stream>>>(kw, e->f32.omega, (size_t)nd * (n + 1)); e->launches++;
    k_convert<double, float><<<1, 256, 0, e->stream>>>(e->f64.omega2, e->f32.omega2, (size_t)nd * (n + 1));
    e->launches++;
    // uniform p, zero D
    k_fill<float><<<grid_for(nd * N, 256), 256, 0, e->stream>>>(e->f32.p, nd * N, (float)std::ldexp(1.0, -n)); e->launches++;
    k_fill<double><<<grid_for(nd * N, 256), 256, 0, e->stream>>>(e->f64.p, nd * N, std::ldexp(1.0, -n)); e->launches++;
    k_fill<float><<<grid_for(nd * N, 256), 256, 0, e->stream>>>(e->f32.D, nd * N, 0.0f); e->launches++;
    k_fill<double><<<grid_for(nd * N, 256), 256, 0, e->stream>>>(e->f64.D, nd * N, 0.0); e->launches++;
    if (e->opt.enable_literal) {
        BDC_TRY(upload_literal_tables(e));
        k_fill<double><<<grid_for(nd * N, 256), 256, 0, e->stream>>>(e->lit_p, nd * N, std::ldexp(1.0, -n)); e->launches++;
        k_fill<double><<<grid_for((size_t)nd * e->R, 256), 256, 0, e->stream>>>(e->lit_D, (size_t)nd * e->R, 0.0); e->launches++;
        k_fill<double><<<grid_for(nd * M, 256), 256, 0, e->stream>>>(e->lit_q, nd * M, 0.0); e->launches++;
    }
    BDC_CUDA_TRY(cudaGetLastError());
    BDC_TRY(sweep_prepare<float>(e, e->f32));
    BDC_TRY(sweep_prepare<double>(e, e->f64));
    BDC_TRY(sync_check(e, "bdc_bind precompute"));
    {
        // a status recorded by the precompute (the checked build's index checks)
        std::vector<double> h;
        BDC_TRY(read_inst(e, h));
        for (int z = 0; z < nd; z++)
            if (h[(size_t)z * INST_STRIDE + I_STATUS] != 0.0)
                BDC_FAIL((bdc_status)(int)h[(size_t)z * INST_STRIDE + I_STATUS], "bdc_bind: the precompute recorded a failure");
    }
    e->cur = 0;
    e->bound = true;
    return BDC_OK;
}

// ---------------------------------------------------------------------------
// representations of p: 0 = FP32 sweep, 1 = FP64 sweep, 2 = literal (FP64)
// ---------------------------------------------------------------------------
// complement half mode left: rebuild the upper half of p and D
static bdc_status unhalf(bdc_engine *e) {
    // half-mode iterations leave D un-averaged (the next forward pass averages
    // it on the fly): average the current precision's D before mirroring
    const bool sym = e->opt.symmetrize && e->orbit_ok;
    if (sym && e->cur == 0 && e->half_active[0]) BDC_TRY(launch_symmetrize<float>(e, e->f32.D, e->half_n2[0]));
    if (sym && e->cur == 1 && e->half_active[1]) BDC_TRY(launch_symmetrize<double>(e, e->f64.D, e->half_n2[1]));
    if (e->half_active[0] || e->half_active[1]) e->f1_current[0] = e->f1_current[1] = false;
    if (e->half_active[0]) {
        BDC_TRY(launch_mirror_half<float>(e, e->f32.p, e->half_n2[0]));
        BDC_TRY(launch_mirror_half<float>(e, e->f32.D, e->half_n2[0]));
        e->half_active[0] = false;
    }
    if (e->half_active[1]) {
        BDC_TRY(launch_mirror_half<double>(e, e->f64.p, e->half_n2[1]));
        BDC_TRY(launch_mirror_half<double>(e, e->f64.D, e->half_n2[1]));
        e->half_active[1] = false;
    }
    return BDC_OK;
}

// drop the cached graphs of one precision (both impls, both lengths)
static void drop_graphs_prec(bdc_engine *e, int prec) {
    for (int b = 0; b < 2; b++) {
        if (e->graph[prec][b]) {
            cudaGraphExecDestroy(e->graph[prec][b]);
            e->graph[prec][b] = nullptr;
        }
        if (e->graph1[prec][b]) {
            cudaGraphExecDestroy(e->graph1[prec][b]);
            e->graph1[prec][b] = nullptr;
        }
    }
}

static void drop_graphs(bdc_engine *e) {
    for (int a = 0; a < 2; a++) drop_graphs_prec(e, a);
}

static bdc_status materialize(bdc_engine *e) {
    // stepped iterations owe the orbit mean of p (they apply the update without
    // averaging D over orbits): take it now, bit-identical over every orbit
    if (e->cur <= 1 && e->p_unsym[e->cur]) {
        if (e->opt.symmetrize && e->orbit_ok) {
            const int n2h = e->half_active[e->cur] ? e->half_n2[e->cur] : 0;
            if (e->cur == 0) BDC_TRY(launch_symmetrize<float>(e, e->f32.p, n2h, true));
            else BDC_TRY(launch_symmetrize<double>(e, e->f64.p, n2h, true));
        }
        e->p_unsym[e->cur] = false;
    }
    e->f1_current[0] = e->f1_current[1] = false;
    BDC_TRY(unhalf(e));
    BDC_TRY(activate(e, -1.0));
    if (e->cur == 0) return launch_apply_pending<float>(e, e->f32);
    if (e->cur == 1) return launch_apply_pending<double>(e, e->f64);
    BDC_TRY(launch_literal_update(e));  // applies the pending factor to every orbit member
    return launch_clear_pending(e);
}

static bdc_status make_current(bdc_engine *e, int target) {
    if (e->cur == target) return BDC_OK;
    if (target == 2 && !e->opt.enable_literal) BDC_FAIL(BDC_EINVAL, "literal path disabled (enable_literal = 0)");
    BDC_TRY(materialize(e));
    const size_t cnt = (size_t)e->nd << e->n;
    const int g = grid_for(cnt, 256);
    const float *s32 = e->f32.p;
    const double *s64 = (e->cur == 1) ? e->f64.p : e->lit_p;
    if (target == 0) {
        k_convert<double, float><<<g, 256, 0, e->stream>>>(s64, e->f32.p, cnt); e->launches++;
    } else {
        double *dst = (target == 1) ? e->f64.p : e->lit_p;
        if (e->cur == 0) {
            k_convert<float, double><<<g, 256, 0, e->stream>>>(s32, dst, cnt);
            e->launches++;
        } else BDC_CUDA_TRY(cudaMemcpyAsync(dst, s64, cnt * sizeof(double), cudaMemcpyDeviceToDevice, e->stream));
    }
    BDC_CUDA_TRY(cudaGetLastError());
    e->cur = target;
    e->p_unsym[0] = e->p_unsym[1] = false;  // the new copy comes from the averaged p
    return BDC_OK;
}

// ---------------------------------------------------------------------------
// iteration
// ---------------------------------------------------------------------------
// Stepped iterations (the adjoint columns pass applies the update and runs
// the next forward columns pass) need F1 to hold the forward columns pass of
// the current p: run that pass alone.  It applies a pending update (with the
// orbit mean of D in half mode), after which nothing is pending.
template <typename T>
static bdc_status prime_step(bdc_engine *e, PrecBuf<T> &b, int prec, bool half) {
    const bool sym = e->opt.symmetrize && e->orbit_ok;
    BDC_TRY(sweep_forward<T>(e, b, b.p, 1, MODE_ITER, half, half && sym, true, false));
    BDC_TRY(launch_clear_pending(e));
    BDC_TRY(launch_clear_symneed(e));
    BDC_TRY(launch_reset_shift(e));
    if (half) {
        e->half_active[prec] = true;
        e->half_n2[prec] = b.s.n2;
    }
    e->f1_current[prec] = true;
    return BDC_OK;
}

static bdc_status ensure_primed(bdc_engine *e, int prec) {
    if (prec == BDC_FP32) {
        PrecBuf<float> &b = e->f32;
        if (step_possible<float>(e, b.s) && !e->f1_current[0])
            return prime_step<float>(e, b, 0, e->opt.use_half && e->half_ok && half_possible(b.s));
    } else {
        PrecBuf<double> &b = e->f64;
        if (step_possible<double>(e, b.s) && !e->f1_current[1])
            return prime_step<double>(e, b, 1, e->opt.use_half && e->half_ok && half_possible(b.s));
    }
    return BDC_OK;
}

template <typename T>
static bdc_status iter_sweep(bdc_engine *e, PrecBuf<T> &b, int prec) {
    // complement half mode while p is complement-invariant
    const bool half = e->opt.use_half && e->half_ok && half_possible(b.s);
    if (!half && e->half_active[prec]) BDC_TRY(unhalf(e));
    const bool sym = e->opt.symmetrize && e->orbit_ok;
    if (step_possible<T>(e, b.s)) {
        if (!e->f1_current[prec]) BDC_TRY(prime_step<T>(e, b, prec, half));
        BDC_TRY(sweep_forward<T>(e, b, b.p, 1, MODE_ITER, half, false, false));
        BDC_TRY(sweep_adjoint<T>(e, b, b.L, b.omega, b.D, MODE_ITER, half, true));
        BDC_TRY(launch_finalize<T>(e, b, MODE_ITER, 0, half ? b.s.nblk_cols / 2 : b.s.nblk_cols, 1));
        e->f1_current[prec] = true;
        e->p_unsym[prec] = true;
        if (half) {
            e->half_active[prec] = true;
            e->half_n2[prec] = b.s.n2;
        }
        return BDC_OK;
    }
    // orbit mean of D: in half mode fused into the next forward pass (and into
    // unhalf), otherwise a pass of its own
    BDC_TRY(sweep_forward<T>(e, b, b.p, 1, MODE_ITER, half, half && sym));
    BDC_TRY(sweep_adjoint<T>(e, b, b.L, b.omega, b.D, MODE_ITER, half));
    BDC_TRY(launch_finalize<T>(e, b, MODE_ITER, 0, half ? b.s.nblk_cols / 2 : b.s.nblk_cols));
    if (sym && !half) BDC_TRY(launch_symmetrize<T>(e, b.D, 0));
    if (half) {
        e->half_active[prec] = true;
        e->half_n2[prec] = b.s.n2;
    }
    return BDC_OK;
}

static bdc_status iter_literal(bdc_engine *e) {
    int g = literal_grid(e);
    BDC_TRY(launch_literal_update(e));
    BDC_TRY(launch_literal_q(e));
    BDC_TRY(launch_literal_D(e));
    BDC_TRY(launch_literal_reduce(e));
    BDC_TRY(launch_finalize_literal(e, g, g));
    return BDC_OK;
}

static bdc_status iter_once(bdc_engine *e, int prec, int impl) {
    if (impl == BDC_LITERAL) return iter_literal(e);
    return prec == BDC_FP32 ? iter_sweep<float>(e, e->f32, 0) : iter_sweep<double>(e, e->f64, 1);
}

// the cached graph of `chunk` iterations (one == false) or of one iteration
static bdc_status get_graph(bdc_engine *e, int prec, int impl, cudaGraphExec_t *out, bool one = false) {
    cudaGraphExec_t &g = one ? e->graph1[prec][impl] : e->graph[prec][impl];
    // a graph of stepped iterations starts from a current F1 (eager, not captured)
    if (impl == BDC_SWEEP) BDC_TRY(ensure_primed(e, prec));
    if (!g) {
        cudaGraph_t graph;
        const int64_t before = e->launches;
        BDC_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        bdc_status st = BDC_OK;
        const int iters = one ? 1 : e->opt.chunk;
        for (int i = 0; i < iters && st == BDC_OK; i++) st = iter_once(e, prec, impl);
        cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
        (one ? e->graph1_kernels : e->graph_kernels)[prec][impl] = e->launches - before;  // recorded, not yet run
        e->launches = before;
        if (st != BDC_OK) return st;
        if (ce != cudaSuccess) BDC_FAIL(BDC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&g, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            g = nullptr;
            BDC_FAIL(BDC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
    }
    *out = g;
    return BDC_OK;
}

extern "C" bdc_status bdc_prepare(bdc_engine *e, int prec, int impl) {
    if (!e) BDC_FAIL(BDC_EINVAL, "bdc_prepare: engine is NULL");
    if (!e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_prepare: no workspace bound");
    if ((prec != BDC_FP32 && prec != BDC_FP64) || (impl != BDC_SWEEP && impl != BDC_LITERAL) ||
        (impl == BDC_LITERAL && prec != BDC_FP64))
        BDC_FAIL(BDC_EINVAL, "bdc_prepare: bad precision or impl");
    if (impl == BDC_LITERAL && !e->orbit_ok)
        BDC_FAIL(BDC_EINVAL, "bdc_prepare: the literal path needs an orbit-invariant p");
    BDC_TRY(make_current(e, impl == BDC_LITERAL ? 2 : prec));
    if (e->opt.use_graph && e->stream != nullptr) {
        cudaGraphExec_t g;
        BDC_TRY(get_graph(e, prec, impl, &g));
        if (e->opt.chunk > 1) BDC_TRY(get_graph(e, prec, impl, &g, true));
    }
    return sync_check(e, "bdc_prepare");
}

extern "C" bdc_status bdc_ba_iterate(bdc_engine *e, int max_iters, double tol, int prec, int impl, double *lower,
                                     double *upper, int *iters_done) {
    if (!e) BDC_FAIL(BDC_EINVAL, "bdc_ba_iterate: engine is NULL");
    if (!e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_ba_iterate: no workspace bound");
    if (max_iters < 0 || (prec != BDC_FP32 && prec != BDC_FP64) || (impl != BDC_SWEEP && impl != BDC_LITERAL))
        BDC_FAIL(BDC_EINVAL, "bdc_ba_iterate: bad max_iters, precision or impl");
    if (impl == BDC_LITERAL && prec != BDC_FP64) BDC_FAIL(BDC_EINVAL, "bdc_ba_iterate: the literal path is FP64 only");
    if (impl == BDC_LITERAL && !e->orbit_ok)
        BDC_FAIL(BDC_EINVAL, "bdc_ba_iterate: the literal path works on orbit representatives and needs an "
                             "orbit-invariant p (complement and reversal)");
    BDC_TRY(make_current(e, impl == BDC_LITERAL ? 2 : prec));
    BDC_TRY(activate(e, tol));
    const bool graph = e->opt.use_graph && e->stream != nullptr;
    int done = 0;
    std::vector<double> h;
    while (done < max_iters) {
        int c = std::min(e->opt.chunk, max_iters - done);
        if (graph && c == e->opt.chunk) {
            cudaGraphExec_t g;
            BDC_TRY(get_graph(e, prec, impl, &g));
            BDC_CUDA_TRY(cudaGraphLaunch(g, e->stream));
            e->launches += e->graph_kernels[prec][impl];
        } else if (graph) {
            // fewer than `chunk` iterations: the one-iteration graph, c times
            cudaGraphExec_t g;
            BDC_TRY(get_graph(e, prec, impl, &g, true));
            for (int i = 0; i < c; i++) {
                BDC_CUDA_TRY(cudaGraphLaunch(g, e->stream));
                e->launches += e->graph1_kernels[prec][impl];
            }
        } else {
            for (int i = 0; i < c; i++) BDC_TRY(iter_once(e, prec, impl));
        }
        done += c;
        if (tol >= 0.0 && done < max_iters) {
            BDC_TRY(read_inst(e, h));
            bool any = false;
            for (int z = 0; z < e->nd; z++) any |= h[(size_t)z * INST_STRIDE + I_ACTIVE] != 0.0;
            if (!any) break;
        }
    }
    BDC_TRY(read_inst(e, h));
    bdc_status st = BDC_OK;
    for (int z = 0; z < e->nd; z++) {
        const double *I = &h[(size_t)z * INST_STRIDE];
        if (lower) lower[z] = I[I_LOWER];
        if (upper) upper[z] = I[I_UPPER];
        if (iters_done) iters_done[z] = (int)I[I_ITERS];
        if (I[I_STATUS] != 0.0) st = (bdc_status)(int)I[I_STATUS];
    }
    e->iters_total += done;
    if (st == BDC_ETIMEOUT) bdc_set_error("bdc_ba_iterate: a bounded device wait gave up (instance stopped)");
    else if (st == BDC_ECHECK) bdc_set_error("bdc_ba_iterate: an index check of the checked build failed (instance stopped)");
    else if (st != BDC_OK) bdc_set_error("bdc_ba_iterate: non-finite value in a reduction (instance stopped)");
    return st;
}

// ---------------------------------------------------------------------------
// batches: several engines (different n, each with its d values) iterated by
// one CUDA graph; each engine's kernels run on a stream forked from the
// batch stream, so small instances overlap.
// ---------------------------------------------------------------------------
struct bdc_batch {
    std::vector<bdc_engine *> engs;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t main = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    std::vector<int> half_state[2];  // engines' complement-half decisions baked into each graph
    int chunk = 8;
};

extern "C" bdc_status bdc_batch_create(bdc_engine *const *engs, int count, int chunk, bdc_batch **out) {
    if (!out || !engs || count < 1) BDC_FAIL(BDC_EINVAL, "bdc_batch_create: need engines");
    *out = nullptr;
    for (int i = 0; i < count; i++) {
        if (!engs[i] || !engs[i]->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_batch_create: every engine must be bound");
        if (engs[i]->stream != engs[0]->stream || engs[0]->stream == nullptr)
            BDC_FAIL(BDC_EINVAL, "bdc_batch_create: engines must share one non-default stream");
        for (int j = 0; j < i; j++)
            if (engs[j] == engs[i]) BDC_FAIL(BDC_EINVAL, "bdc_batch_create: an engine appears twice");
    }
    bdc_batch *b = new bdc_batch();
    b->engs.assign(engs, engs + count);
    b->main = engs[0]->stream;
    b->chunk = chunk < 1 ? 1 : chunk;
    b->side.resize(count);
    b->join.resize(count);
    cudaError_t err = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < count && err == cudaSuccess; i++) {
        err = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (err != cudaSuccess) {
        bdc_set_error(std::string("bdc_batch_create: ") + cudaGetErrorString(err));
        delete b;
        return BDC_ECUDA;
    }
    *out = b;
    return BDC_OK;
}

extern "C" void bdc_batch_destroy(bdc_batch *b) {
    if (!b) return;
    for (int p = 0; p < 2; p++)
        if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
    for (size_t i = 0; i < b->side.size(); i++) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

static bdc_status batch_graph(bdc_batch *b, int prec, cudaGraphExec_t *out) {
    std::vector<int> hs;
    for (bdc_engine *e : b->engs) hs.push_back(e->half_ok ? 1 : 0);
    if (b->graph[prec] && hs != b->half_state[prec]) {
        cudaGraphExecDestroy(b->graph[prec]);
        b->graph[prec] = nullptr;
    }
    b->half_state[prec] = hs;
    if (!b->graph[prec]) {
        cudaGraph_t graph;
        std::vector<int64_t> before(b->engs.size());
        for (bdc_engine *e : b->engs) BDC_TRY(ensure_primed(e, prec));
        BDC_CUDA_TRY(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
        bdc_status st = BDC_OK;
        cudaError_t ce = cudaEventRecord(b->fork, b->main);
        for (size_t i = 0; i < b->engs.size() && st == BDC_OK && ce == cudaSuccess; i++) {
            bdc_engine *e = b->engs[i];
            ce = cudaStreamWaitEvent(b->side[i], b->fork, 0);
            before[i] = e->launches;
            e->stream = b->side[i];
            for (int k = 0; k < b->chunk && st == BDC_OK; k++) st = iter_once(e, prec, BDC_SWEEP);
            e->stream = b->main;
            if (ce == cudaSuccess) ce = cudaEventRecord(b->join[i], b->side[i]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->main, b->join[i], 0);
        }
        cudaError_t ce2 = cudaStreamEndCapture(b->main, &graph);
        int64_t kernels = 0;
        for (size_t i = 0; i < b->engs.size(); i++) {
            kernels += b->engs[i]->launches - before[i];
            b->engs[i]->launches = before[i];
        }
        if (st != BDC_OK) return st;
        if (ce != cudaSuccess || ce2 != cudaSuccess)
            BDC_FAIL(BDC_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
        ce = cudaGraphInstantiate(&b->graph[prec], graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            b->graph[prec] = nullptr;
            BDC_FAIL(BDC_ECUDA, std::string("batch instantiate: ") + cudaGetErrorString(ce));
        }
        b->graph_kernels[prec] = kernels;
    }
    *out = b->graph[prec];
    return BDC_OK;
}

extern "C" bdc_status bdc_batch_iterate(bdc_batch *b, int max_iters, double tol, int prec, int *iters_launched) {
    if (!b) BDC_FAIL(BDC_EINVAL, "bdc_batch_iterate: batch is NULL");
    if (max_iters < 0 || (prec != BDC_FP32 && prec != BDC_FP64)) BDC_FAIL(BDC_EINVAL, "bdc_batch_iterate: bad arguments");
    for (bdc_engine *e : b->engs) {
        BDC_TRY(make_current(e, prec));
        BDC_TRY(activate(e, tol));
    }
    cudaGraphExec_t g;
    BDC_TRY(batch_graph(b, prec, &g));
    int done = 0;
    std::vector<double> h;
    while (done < max_iters) {
        for (bdc_engine *e : b->engs) BDC_TRY(ensure_primed(e, prec));
        BDC_CUDA_TRY(cudaGraphLaunch(g, b->main));
        b->engs[0]->launches += b->graph_kernels[prec];
        done += b->chunk;
        if (tol >= 0.0 && done < max_iters) {
            bool any = false;
            for (bdc_engine *e : b->engs) {
                BDC_TRY(read_inst(e, h));
                for (int z = 0; z < e->nd; z++) any |= h[(size_t)z * INST_STRIDE + I_ACTIVE] != 0.0;
            }
            if (!any) break;
        }
    }
    BDC_CUDA_TRY(cudaStreamSynchronize(b->main));
    for (bdc_engine *e : b->engs) e->iters_total += done;
    if (iters_launched) *iters_launched = done;
    bdc_status st = BDC_OK;
    for (bdc_engine *e : b->engs) {
        BDC_TRY(read_inst(e, h));
        for (int z = 0; z < e->nd; z++)
            if (h[(size_t)z * INST_STRIDE + I_STATUS] != 0.0) st = (bdc_status)(int)h[(size_t)z * INST_STRIDE + I_STATUS];
    }
    if (st == BDC_ETIMEOUT) bdc_set_error("bdc_batch_iterate: a bounded device wait gave up (instance stopped)");
    else if (st != BDC_OK) bdc_set_error("bdc_batch_iterate: non-finite value in a reduction (instance stopped)");
    return st;
}

extern "C" bdc_status bdc_get_history(bdc_engine *e, int inst, double *lower, double *upper, int len, int *count) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_get_history: no workspace bound");
    if (inst < 0 || inst >= e->nd || len < 0) BDC_FAIL(BDC_EINVAL, "bdc_get_history: bad instance or length");
    std::vector<double> h, lo(BDC_HIST), up(BDC_HIST);
    BDC_TRY(read_inst(e, h));
    long total = (long)h[(size_t)inst * INST_STRIDE + I_HISTN];
    BDC_CUDA_TRY(cudaMemcpy(lo.data(), e->hist + (size_t)inst * 2 * BDC_HIST, BDC_HIST * sizeof(double),
                            cudaMemcpyDeviceToHost));
    BDC_CUDA_TRY(cudaMemcpy(up.data(), e->hist + ((size_t)inst * 2 + 1) * BDC_HIST, BDC_HIST * sizeof(double),
                            cudaMemcpyDeviceToHost));
    long avail = std::min<long>(total, BDC_HIST);
    long m = std::min<long>(avail, len);
    for (long i = 0; i < m; i++) {
        long t = total - m + i;
        if (lower) lower[i] = lo[t % BDC_HIST];
        if (upper) upper[i] = up[t % BDC_HIST];
    }
    if (count) *count = (int)m;
    return BDC_OK;
}

// ---------------------------------------------------------------------------
// divergence and certification
// ---------------------------------------------------------------------------
template <typename T>
static bdc_status divergence_impl(bdc_engine *e, PrecBuf<T> &b, const T *q_dev, double *D_dev) {
    const int nd = e->nd, n = e->n;
    const size_t M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    BDC_TRY(activate(e, -1.0));
    if (!q_dev) {
        BDC_TRY(sweep_forward<T>(e, b, b.p, 0, MODE_DIV));
        BDC_TRY(launch_finalize<T>(e, b, MODE_DIV));  // I_SUMP = log2 sum p
        BDC_TRY(sweep_adjoint<T>(e, b, b.L, b.omega, reinterpret_cast<T *>(D_dev), MODE_DIV));
    } else {
        k_log2_codes_nd<T><<<grid_for(nd * M, 256), 256, 0, e->stream>>>(q_dev, b.aux, M, nd, 0); e->launches++;
        int g = std::min(maxblk, grid_for(M, 256, 1024));
        k_sum_rows<T><<<dim3(g, nd), 256, 0, e->stream>>>(q_dev, M, b.part, maxblk, 1, nullptr, n); e->launches++;
        BDC_CUDA_TRY(cudaGetLastError());
        // q_dev slot 0 is ignored by the sum only if it is 0; the ABI says slot 0 is unused (0)
        PrecBuf<T> tmp = b;
        tmp.s.nblk_cols = g;
        BDC_TRY(launch_finalize<T>(e, tmp, MODE_DIV, 1));  // log2 sum q - h(b)
        BDC_TRY(sweep_adjoint<T>(e, b, b.aux, b.omega, reinterpret_cast<T *>(D_dev), MODE_DIV));
    }
    return BDC_OK;
}

extern "C" bdc_status bdc_divergence(bdc_engine *e, const void *q_dev, int prec, double *D_dev) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_divergence: no workspace bound");
    if (!D_dev || (prec != BDC_FP32 && prec != BDC_FP64)) BDC_FAIL(BDC_EINVAL, "bdc_divergence: bad arguments");
    if (!q_dev) BDC_TRY(make_current(e, prec));
    if (!q_dev) BDC_TRY(materialize(e));
    bdc_status st = (prec == BDC_FP32) ? divergence_impl<float>(e, e->f32, (const float *)q_dev, D_dev)
                                       : divergence_impl<double>(e, e->f64, (const double *)q_dev, D_dev);
    BDC_TRY(st);
    return sync_check(e, "bdc_divergence");
}

extern "C" bdc_status bdc_certify_upper(bdc_engine *e, const double *q_dev, double *upper, double *margin,
                                        double *lower) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_certify_upper: no workspace bound");
    const int nd = e->nd, n = e->n;
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;
    const int maxblk = part_maxblk(e);
    PrecBuf<double> &b = e->f64;
    BDC_TRY(materialize(e));
    BDC_TRY(activate(e, -1.0));
    const double *Lsrc;
    // complement half mode when the certified input is exactly complement-
    // invariant (checked bitwise): q~ is then exactly invariant too (its H1
    // codes are computed and mirrored), so D(cpl x) = D(x) for the q~ used and
    // the max over the stored half of the inputs is the max over all of them;
    // the lower bound's two sums cover the same half (a ratio)
    bool half = false;
    int g0 = std::min(maxblk, grid_for(M, 256, 1024));
    double per_thread = std::ceil((double)M / ((double)g0 * 256.0));
    double Kterms = per_thread + 8.0 + g0;
    if (!q_dev) {
        // p~ = (1 - eps) p / sum p + eps * uniform, in FP64
        int gs = std::min(maxblk, grid_for(N, 256, 1024));
        PrecBuf<double> tmp = b;
        tmp.s.nblk_cols = gs;
        if (e->cur == 0) {
            k_sum_rows<float><<<dim3(gs, nd), 256, 0, e->stream>>>(e->f32.p, N, b.part, maxblk, 0, nullptr, n); e->launches++;
            BDC_TRY(launch_finalize<double>(e, tmp, MODE_DIV));
            k_make_pcert<float><<<grid_for(N, 256), 256, 0, e->stream>>>(n, nd, e->f32.p, e->inst,
                                                                          e->opt.certify_mix, e->pcert); e->launches++;
        } else {
            const double *src = (e->cur == 1) ? e->f64.p : e->lit_p;
            k_sum_rows<double><<<dim3(gs, nd), 256, 0, e->stream>>>(src, N, b.part, maxblk, 0, nullptr, n); e->launches++;
            BDC_TRY(launch_finalize<double>(e, tmp, MODE_DIV));
            k_make_pcert<double><<<grid_for(N, 256), 256, 0, e->stream>>>(n, nd, src, e->inst, e->opt.certify_mix,
                                                                           e->pcert); e->launches++;
        }
        BDC_CUDA_TRY(cudaGetLastError());
        if (e->opt.use_half && half_possible(b.s)) {
            std::vector<uint32_t> flags(nd);
            BDC_CUDA_TRY(cudaMemsetAsync(e->pflags, 0, nd * sizeof(uint32_t), e->stream));
            k_check_cpl<<<dim3(grid_for(N / 2, 256, 1024), nd), 256, 0, e->stream>>>(n, e->pcert, e->pflags);
            e->launches++;
            BDC_CUDA_TRY(cudaGetLastError());
            BDC_CUDA_TRY(cudaMemcpyAsync(flags.data(), e->pflags, nd * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                         e->stream));
            BDC_TRY(sync_check(e, "bdc_certify_upper"));
            half = true;
            for (int z = 0; z < nd; z++) half = half && flags[z] == 0u;
        }
        BDC_TRY(sweep_forward<double>(e, b, e->pcert, 0, MODE_CERT, half));  // q_k and L = log2 min(q_k, 1)
        k_sum_rows<double><<<dim3(g0, nd), 256, 0, e->stream>>>(b.q, M, b.part, maxblk, 2, e->bk, n); e->launches++;
        Lsrc = b.L;
    } else {
        k_check_given_q<<<dim3(grid_for(M, 256, 1024), nd), 256, 0, e->stream>>>(q_dev, M, e->inst); e->launches++;
        k_log2_codes_nd<double><<<grid_for(nd * M, 256), 256, 0, e->stream>>>(q_dev, b.aux, M, nd, 1); e->launches++;
        k_sum_rows<double><<<dim3(g0, nd), 256, 0, e->stream>>>(q_dev, M, b.part, maxblk, 2, nullptr, n); e->launches++;
        Lsrc = b.aux;
    }
    BDC_CUDA_TRY(cudaGetLastError());
    BDC_TRY(sweep_adjoint<double>(e, b, Lsrc, b.omega, e->marg, MODE_CERT, half));
    k_finalize_cert<<<nd, FIN_THREADS, 0, e->stream>>>(nd, b.part, maxblk, g0, half ? b.s.nblk_cols / 2 : b.s.nblk_cols,
                                                       Kterms, q_dev ? 0 : 1, e->inst); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    std::vector<double> h;
    BDC_TRY(read_inst(e, h));
    bdc_status st = BDC_OK;
    for (int z = 0; z < nd; z++) {
        const double *I = &h[(size_t)z * INST_STRIDE];
        if (upper) upper[z] = I[I_CERT_U];
        if (margin) margin[z] = I[I_CERT_M];
        if (lower) lower[z] = I[I_CERT_LO];
        if (I[I_STATUS] != 0.0 && st != BDC_ENONFINITE) st = (bdc_status)(int)I[I_STATUS];
    }
    if (st == BDC_EINVAL) bdc_set_error("bdc_certify_upper: the given q must be positive at every code");
    else if (st != BDC_OK) bdc_set_error("bdc_certify_upper: non-finite value (in the given q or the certified bound)");
    return st;
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
// current p (after the pending update), unnormalised, as doubles
static bdc_status download_p(bdc_engine *e, double *p_host, bool normalize) {
    BDC_TRY(materialize(e));
    const size_t N = (size_t)1 << e->n, cnt = N * e->nd;
    if (e->cur == 0) {
        std::vector<float> tmp(cnt);
        BDC_CUDA_TRY(cudaMemcpyAsync(tmp.data(), e->f32.p, cnt * sizeof(float), cudaMemcpyDeviceToHost, e->stream));
        BDC_TRY(sync_check(e, "download p"));
        for (size_t i = 0; i < cnt; i++) p_host[i] = tmp[i];
    } else {
        const double *src = (e->cur == 1) ? e->f64.p : e->lit_p;
        BDC_CUDA_TRY(cudaMemcpyAsync(p_host, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
        BDC_TRY(sync_check(e, "download p"));
    }
    if (normalize)
        for (int z = 0; z < e->nd; z++) {
            double s = 0.0;
            for (size_t x = 0; x < N; x++) s += p_host[z * N + x];
            for (size_t x = 0; x < N; x++) p_host[z * N + x] /= s;
        }
    return BDC_OK;
}

// set p of every representation (FP64 copy exact; FP32 rounded), no pending
// update.  The host array is copied into a scratch area of the workspace and
// checked there on the device (finite, non-negative, positive sum, and the
// invariances the half mode, the orbit mean and the literal path rely on);
// only a valid p replaces the engine's.
static bdc_status upload_p(bdc_engine *e, const double *p_host, bool normalize) {
    const int n = e->n, nd = e->nd;
    const size_t N = (size_t)1 << n, cnt = N * nd;
    const int maxblk = part_maxblk(e);
    double *scratch = e->marg;  // [nd][2^n] doubles, free between calls
    double *part = e->f64.part;
    const int nb = std::min(maxblk, grid_for(N, 256, 1024));
    BDC_CUDA_TRY(cudaMemcpyAsync(scratch, p_host, cnt * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    BDC_CUDA_TRY(cudaMemsetAsync(e->pflags, 0, nd * sizeof(uint32_t), e->stream));
    k_check_p<<<dim3(nb, nd), 256, 0, e->stream>>>(n, scratch, e->pflags, part, maxblk); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    std::vector<uint32_t> flags(nd);
    std::vector<double> sums((size_t)nd * nb);
    BDC_CUDA_TRY(cudaMemcpyAsync(flags.data(), e->pflags, nd * sizeof(uint32_t), cudaMemcpyDeviceToHost, e->stream));
    for (int z = 0; z < nd; z++)
        BDC_CUDA_TRY(cudaMemcpy2DAsync(sums.data() + (size_t)z * nb, sizeof(double),
                                       part + (size_t)z * 2 * maxblk * 4, 4 * sizeof(double), sizeof(double), nb,
                                       cudaMemcpyDeviceToHost, e->stream));
    BDC_TRY(sync_check(e, "bdc_set_p checks"));
    bool sym = true, orb = true;
    for (int z = 0; z < nd; z++) {
        if (flags[z] & 1u) BDC_FAIL(BDC_EINVAL, "bdc_set_p: entries must be finite and non-negative");
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += sums[(size_t)z * nb + b];
        if (!(s > 0.0) || !std::isfinite(s)) BDC_FAIL(BDC_EINVAL, "bdc_set_p: every instance needs a positive sum");
        sym = sym && !(flags[z] & 2u);
        orb = orb && !(flags[z] & 4u);
    }
    if (normalize) {
        k_normalize_p<<<dim3(grid_for(N, 256, 1024), nd), FIN_THREADS, 0, e->stream>>>(n, scratch, part, maxblk, nb);
        e->launches++;
        BDC_CUDA_TRY(cudaGetLastError());
    }
    // complement half mode needs p(x) == p(cpl x) exactly; the orbit mean of D
    // and the literal path (work on orbit representatives) need invariance
    // under reversal too
    orb = orb && sym;
    if (sym != e->half_ok || orb != e->orbit_ok) drop_graphs(e);
    e->half_ok = sym;
    e->orbit_ok = orb;
    e->half_active[0] = e->half_active[1] = false;
    e->f1_current[0] = e->f1_current[1] = false;
    e->p_unsym[0] = e->p_unsym[1] = false;
    BDC_CUDA_TRY(cudaMemcpyAsync(e->f64.p, scratch, cnt * sizeof(double), cudaMemcpyDeviceToDevice, e->stream));
    BDC_TRY(sync_check(e, "bdc_set_p upload"));
    const int g = grid_for(cnt, 256);
    k_convert<double, float><<<g, 256, 0, e->stream>>>(e->f64.p, e->f32.p, cnt); e->launches++;
    if (e->opt.enable_literal)
        BDC_CUDA_TRY(cudaMemcpyAsync(e->lit_p, e->f64.p, cnt * sizeof(double), cudaMemcpyDeviceToDevice, e->stream));
    std::vector<double> h;
    BDC_TRY(read_inst(e, h));
    for (int z = 0; z < e->nd; z++) {
        h[(size_t)z * INST_STRIDE + I_PENDING] = 0.0;
        h[(size_t)z * INST_STRIDE + I_HISTN] = 0.0;
        h[(size_t)z * INST_STRIDE + I_SYMNEED] = 0.0;
    }
    BDC_CUDA_TRY(cudaMemcpyAsync(e->inst, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    e->cur = 1;
    return sync_check(e, "bdc_set_p");
}

extern "C" bdc_status bdc_get_p(bdc_engine *e, double *p_host) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_get_p: no workspace bound");
    if (!p_host) BDC_FAIL(BDC_EINVAL, "bdc_get_p: NULL output");
    return download_p(e, p_host, true);
}

extern "C" bdc_status bdc_set_p(bdc_engine *e, const double *p_host) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_set_p: no workspace bound");
    if (!p_host) BDC_FAIL(BDC_EINVAL, "bdc_set_p: NULL input");
    return upload_p(e, p_host, true);
}

extern "C" bdc_status bdc_get_q(bdc_engine *e, int prec, double *q_host) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_get_q: no workspace bound");
    if (!q_host || (prec != BDC_FP32 && prec != BDC_FP64)) BDC_FAIL(BDC_EINVAL, "bdc_get_q: bad arguments");
    BDC_TRY(make_current(e, prec));
    BDC_TRY(materialize(e));
    BDC_TRY(activate(e, -1.0));
    const int n = e->n, nd = e->nd;
    const size_t M = (size_t)2 << n, cnt = M * nd;
    std::vector<double> qk(cnt);
    if (prec == BDC_FP32) {
        BDC_TRY(sweep_forward<float>(e, e->f32, e->f32.p, 0, MODE_DIV));
        BDC_TRY(launch_finalize<float>(e, e->f32, MODE_DIV));
        std::vector<float> t(cnt);
        BDC_CUDA_TRY(cudaMemcpyAsync(t.data(), e->f32.q, cnt * sizeof(float), cudaMemcpyDeviceToHost, e->stream));
        BDC_TRY(sync_check(e, "bdc_get_q"));
        for (size_t i = 0; i < cnt; i++) qk[i] = t[i];
    } else {
        BDC_TRY(sweep_forward<double>(e, e->f64, e->f64.p, 0, MODE_DIV));
        BDC_TRY(launch_finalize<double>(e, e->f64, MODE_DIV));
        BDC_CUDA_TRY(cudaMemcpyAsync(qk.data(), e->f64.q, cnt * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
        BDC_TRY(sync_check(e, "bdc_get_q"));
    }
    std::vector<double> h, bk((size_t)nd * (n + 1));
    BDC_TRY(read_inst(e, h));
    BDC_CUDA_TRY(cudaMemcpy(bk.data(), e->bk, bk.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int z = 0; z < nd; z++) {
        double inv = std::exp2(-h[(size_t)z * INST_STRIDE + I_SUMP]);
        q_host[z * M] = 0.0;
        for (size_t c = 1; c < M; c++) {
            int k = 63 - __builtin_clzll((unsigned long long)c);
            q_host[z * M + c] = bk[(size_t)z * (n + 1) + k] * qk[z * M + c] * inv;
        }
    }
    return BDC_OK;
}

extern "C" bdc_status bdc_get_q_literal(bdc_engine *e, double *q_host) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_get_q_literal: no workspace bound");
    if (!q_host) BDC_FAIL(BDC_EINVAL, "bdc_get_q_literal: NULL output");
    if (!e->opt.enable_literal) BDC_FAIL(BDC_EINVAL, "bdc_get_q_literal: literal path disabled (enable_literal = 0)");
    if (!e->orbit_ok)
        BDC_FAIL(BDC_EINVAL, "bdc_get_q_literal: the literal path needs an orbit-invariant p (complement and reversal)");
    BDC_TRY(make_current(e, 2));
    BDC_TRY(materialize(e));  // the pending update is applied to every orbit member
    BDC_TRY(activate(e, -1.0));
    BDC_TRY(launch_literal_q(e));  // per-length q_k(y) * sum p, every code of every class
    const int n = e->n, nd = e->nd;
    const size_t N = (size_t)1 << n, M = (size_t)2 << n;
    std::vector<double> qk(M * nd), p(N * nd), bk((size_t)nd * (n + 1));
    BDC_CUDA_TRY(cudaMemcpyAsync(qk.data(), e->lit_q, qk.size() * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(p.data(), e->lit_p, p.size() * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    BDC_CUDA_TRY(cudaMemcpyAsync(bk.data(), e->bk, bk.size() * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    BDC_TRY(sync_check(e, "bdc_get_q_literal"));
    for (int z = 0; z < nd; z++) {
        double s = 0.0;
        for (size_t x = 0; x < N; x++) s += p[z * N + x];
        q_host[z * M] = 0.0;
        for (size_t c = 1; c < M; c++) {
            int k = 63 - __builtin_clzll((unsigned long long)c);
            q_host[z * M + c] = bk[(size_t)z * (n + 1) + k] * qk[z * M + c] / s;
        }
    }
    return BDC_OK;
}

extern "C" int64_t bdc_num_reps(const bdc_engine *e) { return e ? e->R : 0; }
extern "C" int64_t bdc_num_output_classes(const bdc_engine *e) { return e ? e->Rout : 0; }

extern "C" bdc_status bdc_get_rep_stats(bdc_engine *e, int64_t r, uint64_t *x, int *orbit, uint64_t *N_k,
                                        double *S_k) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_get_rep_stats: no workspace bound");
    if (r < 0 || r >= e->R) BDC_FAIL(BDC_EINVAL, "bdc_get_rep_stats: representative index out of range");
    const int n = e->n;
    uint32_t xv;
    uint8_t o;
    std::vector<uint32_t> nk(n + 1);
    BDC_CUDA_TRY(cudaMemcpy(&xv, e->reps + r, sizeof xv, cudaMemcpyDeviceToHost));
    BDC_CUDA_TRY(cudaMemcpy(&o, e->osize + r, sizeof o, cudaMemcpyDeviceToHost));
    BDC_CUDA_TRY(cudaMemcpy(nk.data(), e->Nk + (size_t)r * (n + 1), (n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (S_k) BDC_CUDA_TRY(cudaMemcpy(S_k, e->Sk + (size_t)r * (n + 1), (n + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (x) *x = xv;
    if (orbit) *orbit = o;
    if (N_k)
        for (int k = 0; k <= n; k++) N_k[k] = nk[k];
    return BDC_OK;
}

extern "C" bdc_status bdc_output_classes(bdc_engine *e, int64_t *cls_host) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_output_classes: no workspace bound");
    if (!cls_host) BDC_FAIL(BDC_EINVAL, "bdc_output_classes: NULL output");
    const size_t M = (size_t)2 << e->n;
    std::vector<int32_t> t(M);
    BDC_CUDA_TRY(cudaMemcpy(t.data(), e->ocls, M * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < M; c++) cls_host[c] = (c == 0) ? -1 : t[c];
    return BDC_OK;
}

extern "C" bdc_status bdc_save(bdc_engine *e, const char *path) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_save: no workspace bound");
    if (!path) BDC_FAIL(BDC_EINVAL, "bdc_save: NULL path");
    const size_t N = (size_t)1 << e->n, cnt = N * e->nd;
    std::vector<double> p(cnt);
    BDC_TRY(download_p(e, p.data(), false));  // exact device state: resume is bit-identical
    FILE *f = fopen(path, "wb");
    if (!f) BDC_FAIL(BDC_EINVAL, std::string("bdc_save: cannot open ") + path);
    // format 2: magic, {n, nd, channel kind}, the channel (nd values of d, or
    // nd x (n+1) length weights), iterations, p
    const char magic[8] = {'B', 'D', 'C', 'B', 'A', '0', '0', '2'};
    const bool lengths = !e->blen.empty();
    int32_t hdr[3] = {e->n, e->nd, lengths ? 1 : 0};
    const std::vector<double> &chan = lengths ? e->blen : e->d;
    int64_t it = e->iters_total;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              fwrite(chan.data(), sizeof(double), chan.size(), f) == chan.size() && fwrite(&it, sizeof it, 1, f) == 1 &&
              fwrite(p.data(), sizeof(double), cnt, f) == cnt;
    fclose(f);
    if (!ok) BDC_FAIL(BDC_EINVAL, "bdc_save: write failed");
    return BDC_OK;
}

extern "C" bdc_status bdc_load(bdc_engine *e, const char *path) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_load: no workspace bound");
    if (!path) BDC_FAIL(BDC_EINVAL, "bdc_load: NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) BDC_FAIL(BDC_EINVAL, std::string("bdc_load: cannot open ") + path);
    char magic[8];
    int32_t hdr[3];
    int64_t it = 0;
    const bool lengths = !e->blen.empty();
    const std::vector<double> &chan = lengths ? e->blen : e->d;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "BDCBA002", 8) == 0 && fread(hdr, sizeof hdr, 1, f) == 1 &&
              hdr[0] == e->n && hdr[1] == e->nd && hdr[2] == (lengths ? 1 : 0);
    std::vector<double> c(chan.size());
    const size_t N = (size_t)1 << e->n, cnt = N * e->nd;
    std::vector<double> p(cnt);
    ok = ok && fread(c.data(), sizeof(double), c.size(), f) == c.size() && fread(&it, sizeof it, 1, f) == 1 &&
         fread(p.data(), sizeof(double), cnt, f) == cnt;
    fclose(f);
    if (!ok) BDC_FAIL(BDC_EINVAL, "bdc_load: not a checkpoint of this engine (n, nd, channel kind) or truncated");
    if (memcmp(c.data(), chan.data(), c.size() * sizeof(double)) != 0)
        BDC_FAIL(BDC_EINVAL, "bdc_load: checkpoint has a different channel (d values or length weights)");
    BDC_TRY(upload_p(e, p.data(), false));
    e->iters_total = it;
    return BDC_OK;
}

// ---------------------------------------------------------------------------
// test hook
// ---------------------------------------------------------------------------
extern "C" bdc_status bdc_subseq_counts(int n, const uint64_t *x_dev, int64_t nx, uint64_t *N_dev, double *S_dev,
                                        uint64_t *emb_dev, void *stream) {
    if (n < 1 || n > BDC_MAXN) BDC_FAIL(BDC_EINVAL, "bdc_subseq_counts: n must be in [1, 28]");
    if (!x_dev || nx < 0 || (!N_dev && nx > 0)) BDC_FAIL(BDC_EINVAL, "bdc_subseq_counts: bad arguments");
    if (nx == 0) return BDC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BDC_TRY(subseq_counts_impl(n, x_dev, nx, N_dev, S_dev, emb_dev, st, nullptr));
    cudaError_t err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) BDC_FAIL(BDC_ECUDA, std::string("bdc_subseq_counts: ") + cudaGetErrorString(err));
    return BDC_OK;
}

extern "C" int64_t bdc_launch_count(const bdc_engine *e) { return e ? e->launches : 0; }

extern "C" bdc_status bdc_get_schedule(const bdc_engine *e, int prec, int *n1, int *n2, int *width) {
    if (!e || (prec != BDC_FP32 && prec != BDC_FP64)) BDC_FAIL(BDC_EINVAL, "bdc_get_schedule: bad arguments");
    const Sched &s = (prec == BDC_FP32) ? e->f32.s : e->f64.s;
    if (n1) *n1 = s.n1;
    if (n2) *n2 = s.n2;
    if (width) *width = 1 << s.lw;
    return BDC_OK;
}

template <typename T>
static bdc_status time_sweeps(bdc_engine *e, PrecBuf<T> &b, int reps, float *ms) {
    cudaEvent_t a, z;
    BDC_CUDA_TRY(cudaEventCreate(&a));
    BDC_CUDA_TRY(cudaEventCreate(&z));
    bdc_status st = BDC_OK;
    // one untimed pass (first touch), then `reps` timed forward + adjoint sweeps
    // as a BA iteration runs them (complement half mode where it applies; the
    // stepped columns pass where it applies, without storing its update); p is
    // left as it was, D and F1 are overwritten (the caller materialised p first)
    const bool half = e->opt.use_half && e->half_ok && half_possible(b.s);
    const bool stepped = step_possible<T>(e, b.s);
    for (int r = 0; r <= reps && st == BDC_OK; r++) {
        if (r == 1) cudaEventRecord(a, e->stream);
        st = sweep_forward<T>(e, b, b.p, 0, MODE_ITER, half, false, !stepped || r == 0);
        if (st == BDC_OK) st = sweep_adjoint<T>(e, b, b.L, b.omega, b.D, MODE_ITER, half, stepped, false);
    }
    cudaEventRecord(z, e->stream);
    cudaError_t err = cudaEventSynchronize(z);
    if (st == BDC_OK && err == cudaSuccess) err = cudaEventElapsedTime(ms, a, z);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (st != BDC_OK) return st;
    if (err != cudaSuccess) BDC_FAIL(BDC_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(err));
    *ms /= reps;
    return BDC_OK;
}

template <typename T>
static bdc_status autotune_impl(bdc_engine *e, PrecBuf<T> &b, int prec, int reps, double *best_ms) {
    const int n = e->n;
    const size_t tile = (sizeof(T) == 4) ? 32768 : 16384;
    Sched best = b.s;
    float best_t = 1e30f;
    std::vector<Sched> cands;
    if (n <= 14) {  // one in-CTA pass; the split buffers are not reserved below n = 15
        if (best_ms) *best_ms = 0.0;
        return BDC_OK;
    }
    for (int n2 = std::max(8, n - 14); n2 <= std::min(n - 1, (sizeof(T) == 4) ? 14 : 13); n2++) {
        const int n1 = n - n2;
        for (int lw = 0; lw <= std::min(5, n2); lw++) {
            if (((size_t)2 << n1 << lw) > tile) break;
            Sched s{};
            s.n1 = n1;
            s.n2 = n2;
            s.lw = lw;
            s.nblk_cols = 1 << (n2 - lw);
            cands.push_back(s);
        }
    }
    for (const Sched &s : cands) {
        if (s.nblk_cols > part_maxblk(e)) continue;
        b.s = s;
        float t = 0.f;
        BDC_TRY(time_sweeps<T>(e, b, reps, &t));
        if (t < best_t) {
            best_t = t;
            best = s;
        }
    }
    b.s = best;
    drop_graphs_prec(e, prec);
    if (best_ms) *best_ms = best_t;
    return BDC_OK;
}

extern "C" bdc_status bdc_autotune(bdc_engine *e, int prec, int reps, int n2, int width, double *best_ms) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_autotune: no workspace bound");
    if ((prec != BDC_FP32 && prec != BDC_FP64) || reps < 1) BDC_FAIL(BDC_EINVAL, "bdc_autotune: bad arguments");
    BDC_TRY(make_current(e, prec));
    BDC_TRY(materialize(e));
    BDC_TRY(activate(e, -1.0));
    if (n2 > 0) {
        // set a known schedule (e.g. from a cache) instead of searching
        Sched s = make_sched(e->n, prec == BDC_FP32 ? 4 : 8, n2, width);
        const size_t tile = (prec == BDC_FP32) ? 32768 : 16384;
        if (e->n < 15 || s.n2 < 8 || s.n2 > 14 || ((size_t)2 << s.n1 << s.lw) > tile || ((size_t)2 << s.n2) > tile ||
            s.nblk_cols > part_maxblk(e))
            BDC_FAIL(BDC_EINVAL, "bdc_autotune: schedule outside the reserved buffers (n >= 15, 8 <= n2 <= 14, "
                                 "column and row tiles within shared memory)");
        PrecBuf<float> &f = e->f32;
        PrecBuf<double> &d = e->f64;
        if (prec == BDC_FP32) f.s = s;
        else d.s = s;
        drop_graphs_prec(e, prec);
        if (best_ms) *best_ms = 0.0;
        return BDC_OK;
    }
    if (prec == BDC_FP32) return autotune_impl<float>(e, e->f32, prec, reps, best_ms);
    return autotune_impl<double>(e, e->f64, prec, reps, best_ms);
}

extern "C" bdc_status bdc_profile_iteration(bdc_engine *e, int prec, int impl, int reps, double *stage_ms,
                                            char *names, int names_len, int *nstages) {
    if (!e || !e->bound) BDC_FAIL(BDC_ENOTBOUND, "bdc_profile_iteration: no workspace bound");
    if (reps < 1 || !stage_ms || !nstages || (prec != BDC_FP32 && prec != BDC_FP64) ||
        (impl != BDC_SWEEP && impl != BDC_LITERAL) || (impl == BDC_LITERAL && prec != BDC_FP64))
        BDC_FAIL(BDC_EINVAL, "bdc_profile_iteration: bad arguments");
    BDC_TRY(make_current(e, impl == BDC_LITERAL ? 2 : prec));
    BDC_TRY(activate(e, -1.0));
    if (!e->prof_created) {
        for (int i = 0; i < 32; i++) BDC_CUDA_TRY(cudaEventCreate(&e->prof_ev[i]));
        e->prof_created = true;
    }
    std::vector<double> acc(32, 0.0);
    int ns = 0;
    for (int r = 0; r < reps; r++) {
        e->prof_n = 0;
        stage_mark(e, "start");
        bdc_status st = iter_once(e, prec, impl);
        int m = e->prof_n;
        e->prof_n = -1;
        BDC_TRY(st);
        BDC_TRY(sync_check(e, "bdc_profile_iteration"));
        for (int i = 0; i + 1 < m; i++) {
            float ms = 0.f;
            BDC_CUDA_TRY(cudaEventElapsedTime(&ms, e->prof_ev[i], e->prof_ev[i + 1]));
            acc[i] += ms;
        }
        ns = m - 1;
    }
    std::string all;
    for (int i = 0; i < ns; i++) {
        stage_ms[i] = acc[i] / reps;
        if (i) all += ",";
        all += e->prof_name[i + 1];
    }
    if (names && names_len > 0) {
        strncpy(names, all.c_str(), names_len - 1);
        names[names_len - 1] = 0;
    }
    *nstages = ns;
    return BDC_OK;
}

