// Enumeration kernels: orbit representatives (Appendix A), the
// warp-cooperative walk over the distinct subsequences of an input (Sec. 4:
// N_{x,k}, embedding multiplicities, S_k = sum count*log2 count, and the
// literal per-input divergence of Sec. 3), and the walk over the
// supersequences of an output (Sec. 5: the literal output marginal).
//
// Warp-cooperative subsequence walk.  Lane j holds position j of x.  A trie
// node y carries E_j = #embeddings of y into x whose last symbol sits at x_j.
// With S_j = sum_{j'<j} E_{j'} (exclusive warp scan; S_j = 1 at the root),
// the child y.b has E'_j = [x_j = b] S_j and Count(y.b, x) = sum_j E'_j; the
// child exists (y.b is a subsequence) iff that count is > 0.  This is the
// embedding-count form of the paper's NextPos/Cnt recursion: the lowest lane
// with E'_j > 0 is NextPos of the parent's first embedding, and the walk
// visits the distinct subsequences in lexicographic (unrank) order.
#include "bdc_internal.cuh"

#include <algorithm>
#include <cstring>

namespace {

constexpr int WARPS_PER_CTA = 8;
constexpr int STK = 30;  // >= BDC_MAXN + 2

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane) {
    uint32_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    return s - v;
}

// c*log2(c) as an integer part and a 62-bit fraction, summed exactly in two
// 64-bit integers (the fraction carries into the integer part), so the hot
// loop uses no floating point (FP64 issue is scarce on B300).  Table entries
// (c < 65536) come from long double on the host; larger counts are split
// from FP64 here.  sum_{|y|=k} Count log2 Count <= C(n,k) log2 C(n,k) < 2^28.
constexpr double FRAC_SCALE = 4611686018427387904.0;  // 2^62
constexpr unsigned long long FRAC_ONE = 1ull << 62;
__device__ __forceinline__ void clog2c_fix(uint32_t c, const longlong2 *__restrict__ tab, long long &accI,
                                           unsigned long long &accF) {
    long long I;
    unsigned long long F;
    if (tab != nullptr && c < 65536u) {
        longlong2 t = __ldg(tab + c);
        I = t.x;
        F = (unsigned long long)t.y;
    } else if (c <= 1u) {
        return;
    } else {
        double t = (double)c * log2((double)c);
        double fi = floor(t);
        I = (long long)fi;
        F = __double2ull_rn((t - fi) * FRAC_SCALE);
        if (F >= FRAC_ONE) { F -= FRAC_ONE; I += 1; }
    }
    accI += I;
    accF += F;  // both < 2^62 before the add: no overflow
    if (accF >= FRAC_ONE) { accF -= FRAC_ONE; accI += 1; }
}

// The same value split for summing with 64-bit shared-memory atomics:
// hi = I 2^24 + (F >> 38), lo = F mod 2^38 (units of 2^-62 overall).  Over at
// most C(26,13) < 2^24 nodes of one length, sum hi < 2^53 and sum lo < 2^62, so
// neither overflows and the sums are exact in any order.
__device__ __forceinline__ void clog2c_parts(uint32_t c, const longlong2 *__restrict__ tab, unsigned long long &hi,
                                             unsigned long long &lo) {
    long long I = 0;
    unsigned long long F = 0;
    clog2c_fix(c, tab, I, F);
    hi = ((unsigned long long)I << 24) + (F >> 38);
    lo = F & ((1ull << 38) - 1ull);
}

// ---------------------------------------------------------------------------
// orbit representatives of {0,1}^L (L = n for inputs) : is_rep flags counted
// per block, scanned, then written in increasing order (deterministic).
// ---------------------------------------------------------------------------
constexpr int COMPACT_THREADS = 256;
constexpr int COMPACT_PER_THREAD = 8;
constexpr int COMPACT_TILE = COMPACT_THREADS * COMPACT_PER_THREAD;

// mode 0: inputs of length n (code space x in [0,2^n)); mode 1: output codes
// c in [1, 2^(n+1)) (string of length bitlen(c)-1).
__device__ __forceinline__ bool is_rep_item(uint32_t v, int n, int mode) {
    if (mode == 0) return orbit_rep_dev(v, n, nullptr) == v;
    if (v == 0) return false;
    int k = bitlen32(v) - 1;
    uint32_t y = v ^ (1u << k);
    return orbit_rep_dev(y, k, nullptr) == y;
}

__global__ void k_count_reps(int n, int mode, uint64_t total, uint32_t *blk_counts) {
    __shared__ uint32_t red[COMPACT_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * COMPACT_TILE;
    uint32_t c = 0;
    for (int i = 0; i < COMPACT_PER_THREAD; i++) {
        uint64_t v = base + (uint64_t)i * COMPACT_THREADS + threadIdx.x;
        if (v < total && is_rep_item((uint32_t)v, n, mode)) c++;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < COMPACT_THREADS / 32; w++) s += red[w];
        blk_counts[blockIdx.x] = s;
    }
}

// single-block exclusive scan of nb block counts (sequential per thread chunk)
__global__ void k_scan_counts(uint32_t *cnt, int nb) {
    __shared__ uint32_t part[1024];
    int per = (nb + blockDim.x - 1) / blockDim.x;
    int lo = threadIdx.x * per, hi = min(nb, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; i++) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            uint32_t v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int i = lo; i < hi; i++) {
        uint32_t v = cnt[i];
        cnt[i] = run;
        run += v;
    }
}

__global__ void k_write_reps(int n, int mode, uint64_t total, const uint32_t *blk_off, uint32_t *out,
                             uint8_t *osize, int32_t *cls) {
    __shared__ uint32_t wsum[COMPACT_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * COMPACT_TILE;
    uint32_t run = blk_off[blockIdx.x];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = 0; i < COMPACT_PER_THREAD; i++) {
        uint64_t v = base + (uint64_t)i * COMPACT_THREADS + threadIdx.x;
        bool f = v < total && is_rep_item((uint32_t)v, n, mode);
        uint32_t bal = __ballot_sync(0xffffffffu, f);
        uint32_t before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        uint32_t woff = 0, tot = 0;
        for (int w = 0; w < COMPACT_THREADS / 32; w++) {
            if (w < wid) woff += wsum[w];
            tot += wsum[w];
        }
        if (f) {
            uint32_t idx = run + woff + before;
            out[idx] = (uint32_t)v;
            if (mode == 0) {
                int o;
                orbit_rep_dev((uint32_t)v, n, &o);
                osize[idx] = (uint8_t)o;
            } else {
                cls[v] = (int32_t)idx;
            }
        }
        run += tot;
        __syncthreads();
    }
}

// every output code gets the class index of its representative
__global__ void k_fill_classes(int n, int32_t *cls) {
    uint64_t total = 1ull << (n + 1);
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (uint64_t)gridDim.x * blockDim.x) {
        if (c == 0) { cls[0] = -1; continue; }
        int k = bitlen32((uint32_t)c) - 1;
        uint32_t y = (uint32_t)c ^ (1u << k);
        uint32_t r = orbit_rep_dev(y, k, nullptr);
        if (r != y) cls[c] = cls[(1u << k) | r];
    }
}

// ---------------------------------------------------------------------------
// subsequence walk
// ---------------------------------------------------------------------------
enum { WALK_STATS = 0, WALK_LITERAL_D = 1, WALK_EMIT = 2 };

struct WalkArgs {
    int n;
    int64_t count;              // number of inputs to process
    const uint32_t *xs32;       // inputs (reps) as uint32, or
    const uint64_t *xs64;       // inputs as uint64 (test hook)
    uint32_t *counter;          // dynamic work counter (may be null: static)
    // WALK_STATS
    uint32_t *Nk32; uint64_t *Nk64; double *Sk; int stride;
    const longlong2 *tabfix;    // c*log2(c) split as (integer, fraction * 2^62) for c < 65536
    const double *tab_log2;     // log2(c) for c < 4096
    // WALK_LITERAL_D
    const double *L;            // [nd][2^(n+1)] log2 q_k
    const double *kw;           // [nd][n+1] d^(n-k)(1-d)^k
    const double *lkw;          // [nd][n+1] log2 of kw (or 0 where kw == 0)
    const double *lb;           // [nd][n+1] log2 b_k
    const double *bk;           // [nd][n+1] b_k
    const double *l2c;          // [nd][n+1] log2 C(n,k)
    double *Dout;               // [nd][count]
    const double *inst;
    // WALK_EMIT
    uint64_t *emb;
};

template <int MODE>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32) k_subseq_walk(WalkArgs a) {
    // subtrees spanning at most RZ positions are done in closed form: the 62
    // strings of length 1..5, two per lane
    constexpr int RZ = 5;
    __shared__ uint32_t stkE[WARPS_PER_CTA][STK][32];
    // WALK_STATS: per warp and length, the exact sums of c*log2(c) (hi, lo parts);
    // nodes are buffered 32 at a time (lane i holds the i-th) and folded in by
    // all lanes at once
    __shared__ unsigned long long wacc[MODE == WALK_EMIT ? 1 : WARPS_PER_CTA][BDC_MAXN + 1][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = a.n;
    const int z = blockIdx.y;  // instance (literal D)
    // the strings handled by this lane in closed-form subtrees: z of code
    // lane + 2 (lanes 0..29: every string of length 1..4) and z5 = the 5 bits
    // of the lane (every string of length 5); per string its length and, per
    // symbol b, the bits j (1..length) with z_j = b
    static_assert(RZ == 5, "the lane-to-string map covers lengths 1..5");
    const uint32_t zc = (uint32_t)lane + 2u;
    const int zm = bitlen32(zc) - 1;
    uint32_t zmatch0 = 0u, zmatch1 = 0u, z5match0 = 0u, z5match1 = 0u;
    for (int j = 1; j <= zm && j <= 4; j++) {
        if ((zc >> (zm - j)) & 1u) zmatch1 |= 1u << j;
        else zmatch0 |= 1u << j;
    }
    for (int j = 1; j <= 5; j++) {
        if (((uint32_t)lane >> (5 - j)) & 1u) z5match1 |= 1u << j;
        else z5match0 |= 1u << j;
    }
    const unsigned FULL = 0xffffffffu;
    if (MODE == WALK_LITERAL_D && a.inst[z * INST_STRIDE + I_ACTIVE] == 0.0) return;
    const double *st_z = a.inst ? a.inst + z * INST_STRIDE : nullptr;  // where index checks record
    (void)st_z;
    const double *L = (MODE == WALK_LITERAL_D) ? a.L + ((size_t)z << (n + 1)) : nullptr;
    const double *kw = (MODE == WALK_LITERAL_D) ? a.kw + z * (n + 1) : nullptr;
    if (MODE != WALK_EMIT && lane <= BDC_MAXN) {
        wacc[wid][lane][0] = 0ull;
        wacc[wid][lane][1] = 0ull;
    }
    __syncwarp();
    int64_t item = -1;
    int64_t static_next = (int64_t)blockIdx.x * WARPS_PER_CTA + wid;
    const int64_t static_stride = (int64_t)gridDim.x * WARPS_PER_CTA;
    while (true) {
        if (a.counter) {
            uint32_t v = 0;
            if (lane == 0) v = atomicAdd(a.counter + (MODE == WALK_LITERAL_D ? z : 0), 1u);
            item = __shfl_sync(FULL, v, 0);
        } else {
            item = static_next;
            static_next += static_stride;
        }
        if (item >= a.count) break;
        uint64_t x = a.xs32 ? (uint64_t)a.xs32[item] : a.xs64[item];
        const int xb = (lane < n) ? (int)((x >> (n - 1 - lane)) & 1u) : 2;
        // Az[t] = Count(z, x[i+1:]) at window position i = n - 1 - RZ + t for this
        // lane's string z (A5 likewise for z5), by the suffix DP Cs[j] =
        // #embeddings of z_j..z_zm in the suffix read so far (Cs[zm+1] = 1),
        // prepending x_i: Cs[j] += [z_j = x_i] Cs[j+1]
        uint32_t Az[RZ + 1], A5[RZ + 1];
        {
            uint32_t Cs[RZ + 2], C5[RZ + 2];
#pragma unroll
            for (int j = 1; j <= RZ + 1; j++) {
                Cs[j] = (j == zm + 1) ? 1u : 0u;
                C5[j] = (j == 6) ? 1u : 0u;
            }
            Cs[0] = C5[0] = 0u;
#pragma unroll
            for (int t = RZ; t >= 0; t--) {
                const int i = n - 1 - RZ + t;
                Az[t] = Cs[1];
                A5[t] = C5[1];
                if (i >= 0) {
                    const bool one = (x >> (n - 1 - i)) & 1u;
                    const uint32_t mt = one ? zmatch1 : zmatch0, m5 = one ? z5match1 : z5match0;
#pragma unroll
                    for (int j = 1; j <= RZ; j++) {
                        Cs[j] += ((mt >> j) & 1u) * Cs[j + 1];
                        C5[j] += ((m5 >> j) & 1u) * C5[j + 1];
                    }
                }
            }
        }
        // per-lane accumulators: lane k owns length k (stats) / a 32-slot
        // gather buffer (literal D)
        uint32_t accN = (lane == 0) ? 1u : 0u;
        long long accI = 0;
        unsigned long long accF = 0;
        double accD = 0.0;
        uint32_t bcode = 0, bcnt = 0;
        int nbuf = 0;
        uint32_t stk_code = 0, stk_cnt = 0;  // lane s holds stack slot s
        int sp = 0;
        if (MODE == WALK_EMIT && lane == 0) a.emb[1] = 1;
        if (MODE == WALK_LITERAL_D) {
            // empty output: count 1, weight kw_0 (its count*log2 count is 0)
            double w = kw[0];
            if (lane == 0 && w > 0.0) accD += w * L[1];
        }
        // root children
#pragma unroll
        for (int b = 1; b >= 0; b--) {
            uint32_t E = (xb == b) ? 1u : 0u;
            uint32_t c = __popc(__ballot_sync(FULL, xb == b));
            if (c > 0) {
                if (BDC_IN_RANGE(sp, STK, st_z)) stkE[wid][sp][lane] = E;
                if (lane == sp) { stk_code = 2u | (uint32_t)b; stk_cnt = c; }
                sp++;
            }
        }
        // record one node (code, length kk, count cnt); all lanes call it
        auto record = [&](uint32_t code, int kk, uint32_t cnt) {
            if (MODE == WALK_STATS) {
                if (lane == kk) accN++;
                if (lane == nbuf) { bcode = (uint32_t)kk; bcnt = cnt; }
                if (++nbuf == 32) {
                    unsigned long long hi = 0ull, lo = 0ull;
                    if (bcnt > 1u) clog2c_parts(bcnt, a.tabfix, hi, lo);
                    if (hi | lo) {
                        atomicAdd(&wacc[wid][bcode][0], hi);
                        atomicAdd(&wacc[wid][bcode][1], lo);
                    }
                    nbuf = 0;
                }
            } else if (MODE == WALK_EMIT) {
                if (lane == 0 && BDC_IN_RANGE(code, (size_t)2 << n, st_z)) a.emb[code] = cnt;
            } else {
                // D_x = sum_k [kw_k S_k(x) - b_k log2 C(n,k)] - sum_y kw_|y| Count(y,x) L(y):
                // per node the cross term in FP64 and count*log2(count) in exact
                // fixed point per length, as in the statistics walk
                if (lane == nbuf) { bcode = code; bcnt = cnt; }
                nbuf++;
                if (nbuf == 32) {
                    const int k2 = bitlen32(bcode) - 1;
                    const double w = (double)bcnt * kw[k2];
                    if (w > 0.0 && BDC_IN_RANGE(bcode, (size_t)2 << n, st_z)) accD += w * L[bcode];
                    unsigned long long hi = 0ull, lo = 0ull;
                    if (bcnt > 1u) clog2c_parts(bcnt, a.tabfix, hi, lo);
                    if (hi | lo) {
                        atomicAdd(&wacc[wid][k2][0], hi);
                        atomicAdd(&wacc[wid][k2][1], lo);
                    }
                    nbuf = 0;
                }
            }
        };
        // The whole subtree below a child y' whose embeddings all end at or after
        // position pm, n - 1 - pm <= RZ, in closed form, two descendants per lane:
        // lane l stands for the string z of code l + 2 (every string of length
        // 1..4 in lanes 0..29) and for z5, its 5 bits (every string of length 5);
        // a count Count(y' z, x) = sum_i E[i] Count(z, x[i+1:]) is linear in the
        // embedding-end vector E, with the coefficients Az (A5) of the lane's
        // strings taken once per input; distinct lanes are distinct strings, and
        // a count of 0 means z does not follow y' in x.
        auto subtree = [&](uint32_t ccode, int kc, uint32_t Eb) {
            // E vanishes below the window, and Az / A5 hold the second factor at
            // every window position
            uint32_t cnt = 0u, cnt5 = 0u;
#pragma unroll
            for (int t = 0; t <= RZ; t++) {
                const int i = n - 1 - RZ + t;
                const uint32_t e = __shfl_sync(FULL, Eb, i >= 0 ? i : 0);
                if (i >= 0) {
                    cnt += e * Az[t];
                    cnt5 += e * A5[t];
                }
            }
            const bool valid = lane < 30 && cnt > 0u, valid5 = cnt5 > 0u;
            // one descendant: its code, length and count
            auto leaf = [&](bool ok, uint32_t dcode, int kk, uint32_t c) {
                if (MODE == WALK_STATS) {
                    if (ok && c > 1u) {  // (a count of 1 adds 1 log2 1 = 0)
                        unsigned long long hi, lo;
                        clog2c_parts(c, a.tabfix, hi, lo);
                        if (hi | lo) {
                            atomicAdd(&wacc[wid][kk][0], hi);
                            atomicAdd(&wacc[wid][kk][1], lo);
                        }
                    }
                } else if (MODE == WALK_EMIT) {
                    if (ok && BDC_IN_RANGE(dcode, (size_t)2 << n, st_z)) a.emb[dcode] = c;
                } else {
                    if (ok) {
                        const double w = (double)c * kw[kk];
                        if (w > 0.0 && BDC_IN_RANGE(dcode, (size_t)2 << n, st_z)) accD += w * L[dcode];
                        unsigned long long hi = 0ull, lo = 0ull;
                        if (c > 1u) clog2c_parts(c, a.tabfix, hi, lo);
                        if (hi | lo) {
                            atomicAdd(&wacc[wid][kk][0], hi);
                            atomicAdd(&wacc[wid][kk][1], lo);
                        }
                    }
                }
            };
            if (MODE == WALK_STATS) {
                // lanes 0-1 hold the strings of length 1, 2-5 length 2, 6-13
                // length 3, 14-29 length 4; every lane one of length 5
                const uint32_t bal = __ballot_sync(FULL, valid), bal5 = __ballot_sync(FULL, valid5);
                if (lane == kc + 1) accN += (uint32_t)__popc(bal & 0x3u);
                if (lane == kc + 2) accN += (uint32_t)__popc(bal & 0x3Cu);
                if (lane == kc + 3) accN += (uint32_t)__popc(bal & 0x3FC0u);
                if (lane == kc + 4) accN += (uint32_t)__popc(bal & 0x3FFFC000u);
                if (lane == kc + 5) accN += (uint32_t)__popc(bal5);
            }
            leaf(valid, (ccode << zm) | (zc - (1u << zm)), kc + zm, cnt);
            leaf(valid5, (ccode << 5) | (uint32_t)lane, kc + 5, cnt5);
        };
        while (sp > 0) {
            sp--;
            uint32_t E = stkE[wid][sp][lane];
            uint32_t code = __shfl_sync(FULL, stk_code, sp);
            uint32_t cnt = __shfl_sync(FULL, stk_cnt, sp);
            int k = bitlen32(code) - 1;
            record(code, k, cnt);
            if (k == n) continue;
            uint32_t S = warp_excl_scan(E, lane);
#pragma unroll
            for (int b = 1; b >= 0; b--) {
                uint32_t Eb = (xb == b) ? S : 0u;
                uint32_t cb = __reduce_add_sync(FULL, Eb);
                if (cb > 0) {
                    const int pm = __ffs(__ballot_sync(FULL, Eb != 0u)) - 1;
                    if (n - 1 - pm <= RZ) {
                        // the child's subtree spans the last RZ positions at most:
                        // record it and all its descendants here instead of stacking it
                        record((code << 1) | (uint32_t)b, k + 1, cb);
                        subtree((code << 1) | (uint32_t)b, k + 1, Eb);
                    } else {
                        if (BDC_IN_RANGE(sp, STK, st_z)) stkE[wid][sp][lane] = Eb;
                        if (lane == sp) { stk_code = (code << 1) | (uint32_t)b; stk_cnt = cb; }
                        sp++;
                    }
                }
            }
        }
        if (MODE == WALK_STATS) {
            if (lane < nbuf) {
                unsigned long long hi = 0ull, lo = 0ull;
                if (bcnt > 1u) clog2c_parts(bcnt, a.tabfix, hi, lo);
                if (hi | lo) {
                    atomicAdd(&wacc[wid][bcode][0], hi);
                    atomicAdd(&wacc[wid][bcode][1], lo);
                }
            }
            __syncwarp();
            if (lane <= n) {
                // total = hi 2^38 + lo in units of 2^-62: integer part and 62-bit fraction
                const unsigned long long hi = wacc[wid][lane][0], lo = wacc[wid][lane][1];
                const unsigned long long rest = ((hi & 0xffffffull) << 38) + lo;  // < 2^63
                accI = (long long)(hi >> 24) + (long long)(rest >> 62);
                accF = rest & (FRAC_ONE - 1ull);
                wacc[wid][lane][0] = 0ull;
                wacc[wid][lane][1] = 0ull;
                const bool ok = BDC_IN_RANGE(item, a.count, st_z);
                if (ok && a.Nk32) a.Nk32[item * a.stride + lane] = accN;
                if (ok && a.Nk64) a.Nk64[item * a.stride + lane] = accN;
                if (ok && a.Sk) a.Sk[item * a.stride + lane] = (double)accI + (double)accF * (1.0 / FRAC_SCALE);
            }
            __syncwarp();
        } else if (MODE == WALK_LITERAL_D) {
            if (lane < nbuf) {
                const int k2 = bitlen32(bcode) - 1;
                const double w = (double)bcnt * kw[k2];
                if (w > 0.0 && BDC_IN_RANGE(bcode, (size_t)2 << n, st_z)) accD += w * L[bcode];
                unsigned long long hi = 0ull, lo = 0ull;
                if (bcnt > 1u) clog2c_parts(bcnt, a.tabfix, hi, lo);
                if (hi | lo) {
                    atomicAdd(&wacc[wid][k2][0], hi);
                    atomicAdd(&wacc[wid][k2][1], lo);
                }
            }
            __syncwarp();
            // lane k: kw_k S_k - b_k log2 C(n,k) (S_k from the exact sums)
            double term = 0.0;
            if (lane <= n) {
                const unsigned long long hi = wacc[wid][lane][0], lo = wacc[wid][lane][1];
                const unsigned long long rest = ((hi & 0xffffffull) << 38) + lo;
                const double Sk = (double)((long long)(hi >> 24) + (long long)(rest >> 62)) +
                                  (double)(rest & (FRAC_ONE - 1ull)) * (1.0 / FRAC_SCALE);
                wacc[wid][lane][0] = 0ull;
                wacc[wid][lane][1] = 0ull;
                if (kw[lane] > 0.0) term = kw[lane] * Sk - a.bk[z * (n + 1) + lane] * a.l2c[z * (n + 1) + lane];
            }
            __syncwarp();
            double Dv = term - accD;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) Dv += __shfl_xor_sync(FULL, Dv, o);
            if (lane == 0 && BDC_IN_RANGE(item, a.count, st_z)) a.Dout[(size_t)z * a.count + item] = Dv;
        }
    }
}

// ---------------------------------------------------------------------------
// supersequence walk (literal output marginal).  Work item = (output class
// representative y of length k, first s_k symbols of x).  Lane j in [0, k]
// holds M_j = #embeddings of y_0..y_{j-1} into the current prefix of x
// (M_0 = 1); appending symbol b gives M'_j = M_j + [y_{j-1} = b] M_{j-1}.  A
// prefix of length i stays only if its longest embedded prefix of y, m, has
// m + (n - i) >= k (Lemma num_superseq's supersequences are exactly the
// leaves).  Leaf x contributes p(x) * M_k.
// ---------------------------------------------------------------------------
struct SuperArgs {
    int n;
    int64_t nitems;
    const uint32_t *oreps;      // class representative codes
    const int64_t *koff;        // [n+2] first class index of each length
    const int64_t *ioff;        // [n+2] first item index of each length
    const int *ks;              // [n+1] split bits per length
    const double *p;            // [nd][2^n]
    double *part;               // [nd][nitems]
    const double *inst;
};

__global__ void __launch_bounds__(WARPS_PER_CTA * 32) k_super_walk(SuperArgs a, uint32_t *counter) {
    constexpr int RB = 5;  // levels below the walk, evaluated one leaf per lane (2^RB = 32)
    __shared__ uint32_t stkM[WARPS_PER_CTA][STK][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const int n = a.n;
    const int z = blockIdx.y;
    if (a.inst[z * INST_STRIDE + I_ACTIVE] == 0.0) return;
    const double *inst_z = a.inst + z * INST_STRIDE;  // where index checks record
    (void)inst_z;
    const double *p = a.p + ((size_t)z << n);
    while (true) {
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(counter + z, 1u);
        int64_t item = __shfl_sync(FULL, v, 0);
        if (item >= a.nitems) break;
        int k = 0;
        while (k < n && a.ioff[k + 1] <= item) k++;
        int s = a.ks[k];
        int64_t rel = item - a.ioff[k];
        int64_t cls = a.koff[k] + (rel >> s);
        uint32_t prefix = (uint32_t)(rel & ((1ll << s) - 1));
        uint32_t code = a.oreps[cls];
        uint32_t y = code ^ (1u << k);
        // lane j >= 1 matches y_{j-1}
        int ysym = (lane >= 1 && lane <= k) ? (int)((y >> (k - lane)) & 1u) : 2;
        uint32_t M = (lane == 0) ? 1u : 0u;
        bool alive = true;
        for (int i = 0; i < s; i++) {
            int b = (prefix >> (s - 1 - i)) & 1;
            uint32_t up = __shfl_up_sync(FULL, M, 1);
            if (ysym == b) M += up;
            uint32_t bal = __ballot_sync(FULL, M > 0u && lane <= k);
            int m = 31 - __clz(bal);
            if (m + (n - i - 1) < k) { alive = false; break; }
        }
        double acc = 0.0;
        if (alive) {
            // The last r <= RB levels in closed form, one leaf per lane: lane t
            // appends the r symbols of t (most significant first) to the prefix
            // and carries the window w[j] = M_{k-RB+j}, j = 0..RB, through them:
            // M'_i = M_i + [y_{i-1} = b] M_{i-1}.  After r steps w[RB] = M_k is
            // the leaf's embedding count (0: not a supersequence); a window entry
            // that misses its update from below the window is wrong after one
            // step and the error climbs one entry per step, so it never reaches
            // w[RB] within r <= RB steps.
            // yw[j]: the symbol y_{i-1} of window entry i = k-RB+j (2: none, i <= 0)
            int yw[RB + 1];
#pragma unroll
            for (int j = 0; j <= RB; j++) {
                const int i = k - RB + j;
                yw[j] = (i >= 1) ? (int)((y >> (k - i)) & 1u) : 2;
            }
            const int dstop = (n - RB > s) ? n - RB : s;  // the depth where the closed form takes over
            auto leaves = [&](uint32_t Mv, uint32_t xpre, int r) {
                uint32_t w[RB + 1];
#pragma unroll
                for (int j = 0; j <= RB; j++) {
                    const int i = k - RB + j;
                    w[j] = __shfl_sync(FULL, Mv, i >= 0 ? i : 0);
                    if (i < 0) w[j] = 0u;
                }
#pragma unroll
                for (int st = 0; st < RB; st++) {
                    if (st < r) {
                        const int b = (lane >> (r - 1 - st)) & 1;
#pragma unroll
                        for (int j = RB; j >= 1; j--)
                            if (yw[j] == b) w[j] += w[j - 1];
                    }
                }
                const uint32_t cnt = w[RB];
                const size_t xi = ((size_t)xpre << r) | (uint32_t)lane;
                if (lane < (1 << r) && cnt && BDC_IN_RANGE(xi, (size_t)1 << n, inst_z)) acc += p[xi] * (double)cnt;
            };
            if (dstop == s) {
                leaves(M, prefix, n - s);
            } else {
                // depth-first from depth s down to dstop - 1; lane t holds the next
                // child to try at depth t, stkM[t] the embedding vector of the
                // prefix of length t; a completable child at depth dstop goes to
                // the closed form
                int depth = s;
                uint32_t x = prefix;
                uint32_t nb_lane = 0;
                if (BDC_IN_RANGE(depth, STK, inst_z)) stkM[wid][depth][lane] = M;
                while (true) {
                    int b = (int)__shfl_sync(FULL, nb_lane, depth);
                    if (b > 1) {
                        depth--;
                        x >>= 1;
                        if (depth < s) break;
                        M = stkM[wid][depth][lane];
                        continue;
                    }
                    if (lane == depth) nb_lane = (uint32_t)(b + 1);
                    uint32_t up = __shfl_up_sync(FULL, M, 1);
                    uint32_t Mc = M + ((ysym == b) ? up : 0u);
                    uint32_t bal = __ballot_sync(FULL, Mc > 0u && lane <= k);
                    int m = 31 - __clz(bal);
                    if (m + (n - depth - 1) < k) continue;  // not completable: prune
                    if (depth + 1 == dstop) {
                        leaves(Mc, (x << 1) | (uint32_t)b, n - dstop);
                        continue;
                    }
                    depth++;
                    x = (x << 1) | (uint32_t)b;
                    M = Mc;
                    if (BDC_IN_RANGE(depth, STK, inst_z)) stkM[wid][depth][lane] = M;
                    if (lane == depth) nb_lane = 0;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0 && BDC_IN_RANGE(item, a.nitems, inst_z)) a.part[(size_t)z * a.nitems + item] = acc;
    }
}

// sum the items of every class in order, normalise by C(n,k), write q and
// log2 q to every code of the orbit
__global__ void k_super_reduce(int n, int64_t Rout, const uint32_t *oreps, const int64_t *ioff,
                               const int64_t *koff, const int *ks, const double *part, int64_t nitems,
                               const double *inv_binom, double *q, double *Lq, const double *inst) {
    const int z = blockIdx.y;
    if (inst[z * INST_STRIDE + I_ACTIVE] == 0.0) return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Rout;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t code = oreps[r];
        int k = bitlen32(code) - 1;
        int s = ks[k];
        int64_t first = ioff[k] + ((r - koff[k]) << s);
        double acc = 0.0;
        for (int64_t t = 0; t < (1ll << s); t++) acc += part[(size_t)z * nitems + first + t];
        double qv = acc * inv_binom[k];
        double lv = log2(qv);
        uint32_t y = code ^ (1u << k);
        uint32_t mask = k ? ((1u << k) - 1u) : 0u;
        uint32_t ry = rev_bits(y, k);
        uint32_t mem[4] = {y, y ^ mask, ry, ry ^ mask};
        double *qz = q + ((size_t)z << (n + 1));
        double *lz = Lq + ((size_t)z << (n + 1));
        for (int t = 0; t < 4; t++) {
            uint32_t c = (1u << k) | mem[t];
            qz[c] = qv;
            lz[c] = lv;
        }
    }
}

int64_t count_items_host(int n, const std::vector<int64_t> &Rk, std::vector<int> &ks, std::vector<int64_t> &ioff) {
    ks.assign(n + 1, 0);
    ioff.assign(n + 2, 0);
    for (int k = 0; k <= n; k++) {
        double leaves = 0;
        for (int i = 0; i <= n - k; i++) leaves += binom_d(n, i);
        int s = 0;
        while (s < n - k && leaves / (double)(1ll << s) > 4096.0) s++;
        ks[k] = s;
        ioff[k + 1] = ioff[k] + (Rk[k] << s);
    }
    return ioff[n + 1];
}

}  // namespace

// number of orbit reps of {0,1}^L (Burnside over {id, cpl, rev, cpl rev})
int64_t num_reps_host(int L) {
    if (L == 0) return 1;
    int64_t fix_rev = 1ll << ((L + 1) / 2);
    int64_t fix_crev = (L % 2 == 0) ? (1ll << (L / 2)) : 0;
    return ((1ll << L) + fix_rev + fix_crev) / 4;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static bdc_status compact(bdc_engine *e, int mode, uint32_t *out, uint8_t *osize, int32_t *cls) {
    uint64_t total = (mode == 0) ? (1ull << e->n) : (1ull << (e->n + 1));
    int nb = (int)((total + COMPACT_TILE - 1) / COMPACT_TILE);
    k_count_reps<<<nb, COMPACT_THREADS, 0, e->stream>>>(e->n, mode, total, e->scan_tmp); e->launches++;
    k_scan_counts<<<1, 1024, 0, e->stream>>>(e->scan_tmp, nb); e->launches++;
    k_write_reps<<<nb, COMPACT_THREADS, 0, e->stream>>>(e->n, mode, total, e->scan_tmp, out, osize, cls); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

bdc_status launch_reps(bdc_engine *e) { return compact(e, 0, e->reps, e->osize, nullptr); }

bdc_status launch_output_classes(bdc_engine *e) {
    BDC_TRY(compact(e, 1, e->oreps, nullptr, e->ocls));
    k_fill_classes<<<1024, 256, 0, e->stream>>>(e->n, e->ocls); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

static int walk_grid() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 8;
}

bdc_status launch_subseq_stats(bdc_engine *e) {
    WalkArgs a{};
    a.n = e->n;
    a.count = e->R;
    a.xs32 = e->reps;
    a.counter = e->counter;
    a.Nk32 = e->Nk;
    a.Sk = e->Sk;
    a.stride = e->n + 1;
    a.tabfix = e->tab_fix;
    a.inst = e->inst;  // (instance 0's status receives index-check failures of the checked build)
    BDC_CUDA_TRY(cudaMemsetAsync(e->counter, 0, 64 * sizeof(uint32_t), e->stream));
    k_subseq_walk<WALK_STATS><<<walk_grid(), WARPS_PER_CTA * 32, 0, e->stream>>>(a); e->launches++;
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

// literal D on representatives: Dout[z][r] = sum_y W log2(W / (b_k q_k(y)))
bdc_status launch_literal_D(bdc_engine *e) {
    WalkArgs a{};
    a.n = e->n;
    a.count = e->R;
    a.xs32 = e->reps;
    a.counter = e->counter + 64;
    a.tab_log2 = e->tab_clog + 4096;
    a.L = e->lit_L;
    a.kw = e->bk + (size_t)e->nd * (e->n + 1);
    a.lkw = e->bk + (size_t)2 * e->nd * (e->n + 1);
    a.lb = e->bk + (size_t)3 * e->nd * (e->n + 1);
    a.bk = e->bk;
    a.l2c = e->bk + (size_t)5 * e->nd * (e->n + 1);
    a.tabfix = e->tab_fix;
    a.Dout = e->lit_D;
    a.inst = e->inst;
    BDC_CUDA_TRY(cudaMemsetAsync(e->counter + 64, 0, e->nd * sizeof(uint32_t), e->stream));
    dim3 grid(walk_grid() / 2 > 1 ? walk_grid() / 2 : 1, e->nd);
    k_subseq_walk<WALK_LITERAL_D><<<grid, WARPS_PER_CTA * 32, 0, e->stream>>>(a); e->launches++; stage_mark(e, "literal_D_walk");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

// literal q: item tables live in the literal partial buffer header
struct SuperTables {
    std::vector<int64_t> koff, ioff;
    std::vector<int> ks;
    int64_t nitems;
};

static SuperTables super_tables(int n) {
    SuperTables t;
    std::vector<int64_t> Rk(n + 1);
    for (int k = 0; k <= n; k++) Rk[k] = num_reps_host(k);
    t.koff.assign(n + 2, 0);
    for (int k = 0; k <= n; k++) t.koff[k + 1] = t.koff[k] + Rk[k];
    t.nitems = count_items_host(n, Rk, t.ks, t.ioff);
    return t;
}

int64_t literal_items(int n) { return super_tables(n).nitems; }

// device-side item tables, at the start of the literal partial buffer
struct LitTab {
    int64_t koff[BDC_MAXN + 2];
    int64_t ioff[BDC_MAXN + 2];
    int ks[BDC_MAXN + 2];
    double inv_binom[BDC_MAXN + 2];
};
size_t literal_part_bytes(int n, int nd) {
    return ((sizeof(LitTab) + 255) & ~(size_t)255) + (size_t)nd * (size_t)literal_items(n) * sizeof(double);
}

bdc_status upload_literal_tables(bdc_engine *e) {
    const int n = e->n;
    SuperTables t = super_tables(n);
    LitTab h;
    memset(&h, 0, sizeof h);
    for (int k = 0; k <= n + 1; k++) { h.koff[k] = t.koff[k]; h.ioff[k] = t.ioff[k]; }
    for (int k = 0; k <= n; k++) { h.ks[k] = t.ks[k]; h.inv_binom[k] = 1.0 / binom_d(n, k); }
    BDC_CUDA_TRY(cudaMemcpy(e->lit_part, &h, sizeof h, cudaMemcpyHostToDevice));
    return BDC_OK;
}

bdc_status launch_literal_q(bdc_engine *e) {
    const int n = e->n;
    SuperTables t = super_tables(n);
    LitTab *dt = (LitTab *)e->lit_part;
    double *part = (double *)((char *)e->lit_part + ((sizeof(LitTab) + 255) & ~(size_t)255));
    uint32_t *ctr = e->counter + 64 + e->nd;
    BDC_CUDA_TRY(cudaMemsetAsync(ctr, 0, e->nd * sizeof(uint32_t), e->stream));
    SuperArgs a{};
    a.n = n;
    a.nitems = t.nitems;
    a.oreps = e->oreps;
    a.koff = dt->koff;
    a.ioff = dt->ioff;
    a.ks = dt->ks;
    a.p = e->lit_p;
    a.part = part;
    a.inst = e->inst;
    dim3 grid(walk_grid() / 2 > 1 ? walk_grid() / 2 : 1, e->nd);
    k_super_walk<<<grid, WARPS_PER_CTA * 32, 0, e->stream>>>(a, ctr); e->launches++; stage_mark(e, "literal_q_walk");
    dim3 g2((unsigned)std::min<int64_t>((e->Rout + 255) / 256, 4096), e->nd);
    k_super_reduce<<<g2, 256, 0, e->stream>>>(n, e->Rout, e->oreps, dt->ioff, dt->koff, dt->ks, part,
                                              t.nitems, dt->inv_binom, e->lit_q, e->lit_L, e->inst); e->launches++; stage_mark(e, "literal_q_reduce");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

// ---------------------------------------------------------------------------
// test hook
// ---------------------------------------------------------------------------
bdc_status subseq_counts_impl(int n, const uint64_t *x_dev, int64_t nx, uint64_t *N_dev, double *S_dev,
                              uint64_t *emb_dev, cudaStream_t st, const longlong2 *tab_fix) {
    WalkArgs a{};
    a.n = n;
    a.count = nx;
    a.xs64 = x_dev;
    a.Nk64 = N_dev;
    a.Sk = S_dev;
    a.stride = n + 1;
    a.tabfix = tab_fix;
    int grid = (int)std::min<int64_t>((nx + WARPS_PER_CTA - 1) / WARPS_PER_CTA, walk_grid());
    if (grid < 1) grid = 1;
    k_subseq_walk<WALK_STATS><<<grid, WARPS_PER_CTA * 32, 0, st>>>(a);
    BDC_CUDA_TRY(cudaGetLastError());
    if (emb_dev && nx == 1) {
        BDC_CUDA_TRY(cudaMemsetAsync(emb_dev, 0, (size_t)sizeof(uint64_t) << (n + 1), st));
        a.emb = emb_dev;
        k_subseq_walk<WALK_EMIT><<<1, WARPS_PER_CTA * 32, 0, st>>>(a);
        BDC_CUDA_TRY(cudaGetLastError());
    }
    return BDC_OK;
}
