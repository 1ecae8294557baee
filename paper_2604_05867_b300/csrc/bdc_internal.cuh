// Internal declarations shared by the CUDA translation units of libbdc.
//
// Encoding used throughout (paper Sec. 2.1 indexes strings from 0):
//   x in {0,1}^n is the integer with x_0 as its most significant of n bits;
//   an output y of length k has code (1<<k)|y; slot 0 of code arrays unused.
//
// Sweep index: at level i of a left-to-right pass over the input symbols, the
// pair (u, s) -- u the output produced by x_0..x_{i-1}, s = x_i..x_{n-1} still
// pending -- sits at P = (code(u) << (n-i)) | s.  Every level shares the index
// range [1, 2^(n+1)); the number of deletions so far is delta(P) =
// n + 1 - bitlen(P), independent of the level.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/bdc.h"

#define BDC_MAXN 28
#define BDC_HIST 8192

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void bdc_set_error(const std::string &msg);

#define BDC_CUDA_TRY(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            bdc_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return BDC_ECUDA;                                                           \
        }                                                                               \
    } while (0)

#define BDC_TRY(call)                                                                   \
    do {                                                                                \
        bdc_status s_ = (call);                                                         \
        if (s_ != BDC_OK) return s_;                                                    \
    } while (0)

// ---------------------------------------------------------------------------
// per-instance device scalars (double slots of inst[z * INST_STRIDE + .])
// ---------------------------------------------------------------------------
enum {
    I_ACTIVE = 0,     // 1 while the instance iterates; 0 once its gap < tol
    I_PENDING = 1,    // 1 when p must still be multiplied by 2^{Dbar - SHIFT}
    I_SHIFT = 2,      // log2 of the last Z (the BA normalisation)
    I_LOWER = 3,      // bounds of the last iteration
    I_UPPER = 4,
    I_ZP = 5,         // sum of unnormalised p of the last iteration
    I_TOL = 6,        // gap tolerance for this call
    I_ITERS = 7,      // iterations run in the current call
    I_HISTN = 8,      // total iterations recorded in the history ring
    I_STATUS = 9,     // 0 ok, else a bdc_status (non-finite, ...)
    I_MAXD = 10,      // max_x D_stored of the last iteration
    I_CERT_U = 11,    // certified bound
    I_CERT_M = 12,    // its margin
    I_CERT_LO = 13,   // FP64 lower bound of the certified input
    I_LOG2SQ = 14,    // log2 sum q~ (certify)
    I_LOG2SQ_ERR = 15,
    I_EH = 16,        // certified bound on |Hb^ - Hb|
    I_DUAL_F = 17,
    I_DUAL_MAXD = 18,
    I_DUAL_GD = 19,
    I_DUAL_ZT = 20,   // log-sum-exp of theta over codes
    I_SUMP = 21,
    I_SYMNEED = 22,   // D of the last iteration still needs the orbit mean
    I_NEGH = 23,      // sum_k b_k log2 b_k = -h(b): the length entropy, added when q is a full marginal
    I_DUAL_S = 24,    // sum_x 2^{(D_x - max D)/tau}
    I_DUAL_C0 = 25,   // sum_k rho_k b_k log2 b_k, rho_k = (n-k)/d - k/(1-d)
    I_DUAL_TAU = 26,
    INST_STRIDE = 32
};

// ---------------------------------------------------------------------------
// sweep schedule: x = x1 x2 with |x1| = n1 (columns pass) and |x2| = n2 (rows
// pass); n2 == 0 means a single in-CTA pass over all n symbols.
// ---------------------------------------------------------------------------
struct Sched {
    // n2 < 0: the streaming schedule (one global-memory pass per input
    // symbol), for sizes whose tiles do not fit in shared memory
    int n1, n2, lw;  // lw = log2 of the column tile width
    int nblk_cols;   // CTAs per instance of the columns passes
};

template <typename T>
struct PrecBuf {
    T *p;        // [nd][2^n] unnormalised input distribution
    T *D;        // [nd][2^n] D_x - log2(sum p) of the last iteration (Dbar after symmetrising)
    T *Hb;       // [nd][2^n] sum_k b_k H_k(x)
    T *q;        // [nd][2^(n+1)] q_k(y) = sum_x p(x) Count(y,x) / C(n,k)
    T *L;        // [nd][2^(n+1)] log2 q_k
    T *F1;       // [nd][2^n1 rows][2^n2]   columns-pass output (rows >= 1)
    T *Tm;       // [nd][2^(n1+1)][2^n2]     rows-pass output, codes c2 in [32, 2^n2)
    T *Ts;       // [nd][32][2^(n1+1)]       rows-pass output, codes c2 < 32 (transposed)
    T *Gb;       // [nd][2^(n1+1)][2^n2]     adjoint rows-pass output
    double *part;  // [nd][2][maxblk][4] block partials
    T *omega;    // [nd][n+1] weight applied to L in the adjoint: b_k / C(n,k)
    T *aux;      // [nd][2^(n+1)] spare code-indexed array (dual bound, certify)
    T *pd;       // [nd][2^n] spare input-indexed array (softmax weights of the dual bound)
    T *omega2;   // [nd][n+1] rho_k b_k / C(n,k) (d-derivative of the adjoint weights)
    Sched s;
};

struct bdc_engine {
    int n = 0, nd = 0;
    std::vector<double> d;     // deletion probability per instance (NaN for a length-mixture channel)
    // Length-mixture channels (bdc_create_lengths): per instance the
    // distribution b_k of the output length, [nd][n+1]; empty for BDC_d.
    std::vector<double> blen;
    bdc_options opt;
    size_t ws_bytes = 0;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;

    // d-free precompute
    int64_t R = 0;          // number of input orbit representatives
    int64_t Rout = 0;       // number of output orbit classes (all lengths)
    uint32_t *pflags = nullptr;  // [nd] checks of a p given by bdc_set_p (bit 0 invalid, 1 not cpl-, 2 not rev-invariant)
    uint32_t *reps = nullptr;   // [R] sorted
    uint8_t *osize = nullptr;   // [R]
    uint32_t *Nk = nullptr;     // [R][n+1]
    double *Sk = nullptr;       // [R][n+1]
    uint32_t *oreps = nullptr;  // [Rout] output class representative codes (sorted)
    int32_t *ocls = nullptr;    // [2^(n+1)] code -> class index
    uint32_t *counter = nullptr;  // work counters (16 words)
    uint32_t *scan_tmp = nullptr; // block counts for compaction
    double *bk = nullptr;       // [nd][n+1] b_k (FP64, host-exact)
    double *tab_clog = nullptr; // [8192]: c*log2(c) and log2(c) for c < 4096 (literal path)
    longlong2 *tab_fix = nullptr; // [65536] c*log2(c) = x + y * 2^-62 (x integer part)
    double *inst = nullptr;     // [nd][INST_STRIDE]
    double *hist = nullptr;     // [nd][2][BDC_HIST]
    double *lit_part = nullptr; // literal path partial buffer
    double *lit_q = nullptr;    // [nd][2^(n+1)] literal q (FP64)
    double *lit_L = nullptr;
    double *lit_p = nullptr;    // [nd][2^n] literal-path p (expanded over all x)
    double *lit_D = nullptr;    // [nd][R]
    double *pcert = nullptr;    // [nd][2^n] certify input
    double *marg = nullptr;     // [nd][2^n] spare FP64 array (certify margins / D output)
    double *dual_w = nullptr;   // [nd][n+1] rho_k b_k
    uint64_t max_N = 0;         // max over reps and k of N_{x,k}

    PrecBuf<float> f32;
    PrecBuf<double> f64;

    // graph cache per (precision, impl): `chunk` iterations, and one iteration
    // (calls that ask for fewer than `chunk`)
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t graph1[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int cur = 0;                // representation holding the current p: 0 FP32, 1 FP64, 2 literal
    bool half_ok = true;        // p is complement-invariant (uniform start, BA iterates)
    bool orbit_ok = true;       // p is invariant under complement and reversal
    bool half_active[2] = {false, false};  // upper half of p/D stale in that precision
    bool f1_current[2] = {false, false};   // F1 holds the forward columns pass of the current p
    bool p_unsym[2] = {false, false};      // stepped iterations ran since p was last orbit-averaged
    int half_n2[2] = {0, 0};    // n2 of the schedule the half mode ran with
    int64_t iters_total = 0;
    int64_t launches = 0;       // kernels launched so far (graph replays included)
    int64_t graph_kernels[2][2] = {{0, 0}, {0, 0}};
    int64_t graph1_kernels[2][2] = {{0, 0}, {0, 0}};
    // stage profiling: when prof_n >= 0, each stage boundary records an event
    cudaEvent_t prof_ev[32];
    const char *prof_name[32];
    bool prof_created = false;
    int prof_n = -1;
};

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
Sched make_sched(int n, int elem_bytes, int n2_override, int w_override);
double binom_d(int n, int k);
int64_t num_reps_host(int n);

// enumeration (enum.cu)
bdc_status launch_reps(bdc_engine *e);
bdc_status launch_subseq_stats(bdc_engine *e);
bdc_status launch_output_classes(bdc_engine *e);
bdc_status launch_literal_q(bdc_engine *e);
bdc_status launch_literal_D(bdc_engine *e);

// sweep (sweep.cu)
template <typename T>
bdc_status sweep_prepare(bdc_engine *e, PrecBuf<T> &b);
template <typename T>
bdc_status sweep_forward(bdc_engine *e, PrecBuf<T> &b, const T *p_src, int apply_update, int mode, bool half = false,
                         bool sym_rev = false, bool cols = true, bool rest = true);
template <typename T>
bdc_status sweep_adjoint(bdc_engine *e, PrecBuf<T> &b, const T *Lsrc, const T *omega, T *Dout, int mode,
                         bool half = false, bool step = false, bool keep_p = true);
bool half_possible(const Sched &s);
// the adjoint columns pass can carry the BA update and the next forward
// columns pass (register-resident column kernels apply)
template <typename T>
bool step_possible(const bdc_engine *e, const Sched &s);

// BA glue (ba.cu)
template <typename T>
bdc_status launch_build_Hb(bdc_engine *e, PrecBuf<T> &b);
// level-by-level sweeps through global memory (the streaming schedule, n2 < 0)
template <typename T>
bdc_status stream_forward(bdc_engine *e, PrecBuf<T> &b, const T *p_src, int apply_update, int mode);
template <typename T>
bdc_status stream_adjoint(bdc_engine *e, PrecBuf<T> &b, const T *Lsrc, const T *omega, T *Dout, int mode);
bdc_status launch_build_Hb_w(bdc_engine *e, const double *w, double *out);
template <typename T>
bdc_status launch_finalize(bdc_engine *e, PrecBuf<T> &b, int mode, int add_negh = 0, int nblk = 0, int stepped = 0);
template <typename T>
bdc_status launch_symmetrize(bdc_engine *e, T *D, int n2h = 0, bool force = false);
template <typename T>
bdc_status launch_mirror_half(bdc_engine *e, T *a, int n2);
template <typename T>
bdc_status launch_apply_pending(bdc_engine *e, PrecBuf<T> &b);
bdc_status launch_literal_update(bdc_engine *e);
bdc_status launch_literal_reduce(bdc_engine *e);
bdc_status launch_clear_pending(bdc_engine *e);
bdc_status launch_clear_symneed(bdc_engine *e);
bdc_status launch_reset_shift(bdc_engine *e);
bdc_status launch_finalize_literal(bdc_engine *e, int nblk0, int nblk1);
bdc_status launch_expand_reps(bdc_engine *e, const double *Dr, double *out);
int literal_grid(const bdc_engine *e);
int part_maxblk(const bdc_engine *e);
int64_t literal_items(int n);
size_t literal_part_bytes(int n, int nd);
bdc_status upload_literal_tables(bdc_engine *e);
bdc_status subseq_counts_impl(int n, const uint64_t *x_dev, int64_t nx, uint64_t *N_dev, double *S_dev,
                              uint64_t *emb_dev, cudaStream_t st, const longlong2 *tab_fix);

// record a stage boundary when profiling (no-op otherwise)
inline void stage_mark(bdc_engine *e, const char *name) {
    if (e->prof_n >= 0 && e->prof_n < 32) {
        e->prof_name[e->prof_n] = name;
        cudaEventRecord(e->prof_ev[e->prof_n++], e->stream);
    }
}

// Index checks of the checked build (compiled with -DBDC_CHECKS): a kernel
// tests an index against the extent of the array it addresses; a failing test
// records BDC_ECHECK in the instance status and the access is skipped, so the
// host reads the failure after the call instead of a fault.  The release build
// compiles the tests away.
#ifdef BDC_CHECKS
__device__ __forceinline__ bool bdc_in_range(size_t i, size_t extent, const double *inst_z) {
    if (i < extent) return true;
    if (inst_z) const_cast<double *>(inst_z)[I_STATUS] = (double)BDC_ECHECK;  // (no record without an engine)
    return false;
}
#define BDC_IN_RANGE(i, extent, inst_z) bdc_in_range((size_t)(i), (size_t)(extent), (inst_z))
#else
#define BDC_IN_RANGE(i, extent, inst_z) true
#endif

// modes of the sweep epilogues
enum { MODE_ITER = 0, MODE_CERT = 1, MODE_DIV = 2, MODE_DUAL = 3, MODE_DUAL_D = 4 };

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bitlen32(uint32_t v) { return 32 - __clz(v); }

// instance flags (I_ACTIVE, I_PENDING, I_SYMNEED) hold exactly 1.0 or 0.0;
// testing their bit pattern keeps FP64 instructions out of FP32 kernels
__device__ __forceinline__ bool flag_set(const double *inst, int slot) {
    return __double_as_longlong(inst[slot]) != 0;
}

__device__ __forceinline__ uint32_t rev_bits(uint32_t v, int L) {
    return L == 0 ? 0u : (__brev(v) >> (32 - L));
}

// smallest member of the orbit of s (length L) under complement and reversal
__device__ __forceinline__ uint32_t orbit_rep_dev(uint32_t s, int L, int *osize) {
    uint32_t mask = (L >= 32) ? 0xffffffffu : ((1u << L) - 1u);
    uint32_t a = s, b = s ^ mask, c = rev_bits(s, L), dd = c ^ mask;
    uint32_t m = min(min(a, b), min(c, dd));
    if (osize) {
        int cnt = 1;
        if (b != a) cnt++;
        if (c != a && c != b) cnt++;
        if (dd != a && dd != b && dd != c) cnt++;
        *osize = cnt;
    }
    return m;
}

// Deterministic block reductions of block partials (blockDim.x = NT): thread
// t folds elements t, t+NT, ... in order, then a fixed shuffle tree and an
// in-order sum of the warp results.  Result in thread 0.  Loads bypass L1:
// the partials may come from other CTAs of the running kernel.
constexpr int FIN_THREADS = 256;
template <int NT = FIN_THREADS>
__device__ __forceinline__ double fin_sum(const double *a, int stride, int count, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += NT) s += __ldcg(a + (size_t)i * stride);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; w++) t += red[w];
    return t;
}
template <int NT = FIN_THREADS>
__device__ __forceinline__ double fin_max(const double *a, int stride, int count, double *red) {
    double s = -INFINITY;
    for (int i = threadIdx.x; i < count; i += NT) s = fmax(s, __ldcg(a + (size_t)i * stride));
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = -INFINITY;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; w++) t = fmax(t, red[w]);
    return t;
}

// End of a BA iteration for instance z (all NT threads of the block call it):
// lower = log2 sum_x (p/Zp) 2^{D_x}, upper = max D + log2 Zp, the normaliser
// of the next update, history, stopping test.  stepped: the update was
// applied in the adjoint columns pass (which also summed p into slot 1 [2]),
// so nothing is left pending.
template <int NT>
__device__ __forceinline__ void finalize_instance(int z, const double *part, int maxblk, int nblk0, int nblk1,
                                                  double *inst, double *hist, int stepped, double *red) {
    double *I = inst + z * INST_STRIDE;
    const double *p0 = part + ((size_t)z * 2 + 0) * maxblk * 4;
    const double *p1 = part + ((size_t)z * 2 + 1) * maxblk * 4;
    double Zp = stepped ? fin_sum<NT>(p1 + 2, 4, nblk1, red) : fin_sum<NT>(p0, 4, nblk0, red);
    double ZD = fin_sum<NT>(p1, 4, nblk1, red);
    double mD = fin_max<NT>(p1 + 1, 4, nblk1, red);
    if (threadIdx.x != 0) return;
    if (I[I_STATUS] != 0.0) {
        // a kernel of this iteration failed (e.g. a bounded wait gave up): the
        // instance stops and keeps that status
        I[I_ACTIVE] = 0.0;
        return;
    }
    if (!isfinite(ZD) || !isfinite(mD) || !(Zp > 0.0) || !isfinite(Zp) || !(ZD > 0.0)) {
        I[I_STATUS] = (double)BDC_ENONFINITE;
        I[I_ACTIVE] = 0.0;
        return;
    }
    double lower = log2(ZD);  // D_x = D_stored + log2 Zp
    double upper = mD + log2(Zp);
    I[I_LOWER] = lower;
    I[I_UPPER] = upper;
    I[I_ZP] = Zp;
    I[I_MAXD] = mD;
    I[I_SHIFT] = log2(ZD);
    I[I_PENDING] = stepped ? 0.0 : 1.0;
    I[I_SYMNEED] = stepped ? 0.0 : 1.0;
    I[I_ITERS] += 1.0;
    long h = (long)I[I_HISTN];
    hist[((size_t)z * 2 + 0) * BDC_HIST + (h % BDC_HIST)] = lower;
    hist[((size_t)z * 2 + 1) * BDC_HIST + (h % BDC_HIST)] = upper;
    I[I_HISTN] = (double)(h + 1);
    if (upper - lower < I[I_TOL]) I[I_ACTIVE] = 0.0;
}

template <typename T>
__device__ __forceinline__ T log2_t(T v);
template <>
__device__ __forceinline__ float log2_t<float>(float v) { return __log2f(v); }
template <>
__device__ __forceinline__ double log2_t<double>(double v) { return log2(v); }

template <typename T>
__device__ __forceinline__ T exp2_t(T v);
template <>
__device__ __forceinline__ float exp2_t<float>(float v) { return exp2f(v); }
template <>
__device__ __forceinline__ double exp2_t<double>(double v) { return exp2(v); }
