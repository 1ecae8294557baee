// Factorised output-marginal sweep and its adjoint.
//
// The channel is never stored.  Reading the input symbols left to right, the
// count-weighted state F_i(u, s) = sum_{r in {0,1}^i} p(r s) Count(u, r) obeys
// (Count of a string ending in symbol b either skips b or matches it with the
// last symbol of u):
//     F_{i+1}(u, s') = F_i(u, 0 s') + F_i(u, 1 s') + F_i(u^-, u_last s')
// and F_n(y) = sum_x p(x) Count(y, x) = C(n,k) q_k(y), the output marginal of
// the exact channel BDC_{n,k} (Sec. 2.2).  In the index P = code(u) << (n-i) | s
// the last term is at P itself, so one step is
//     out[P] = in[P] + in[ins0(P)] + in[ins1(P)]      (P < 2^n)
//     out[P] = in[P]                                   (P >= 2^n, no deletion yet)
// where ins_b(P) inserts bit b at position m = n-i-1.  The adjoint step is
//     G_i[Q] = G_{i+1}[Q] + G_{i+1}[cmp(Q)],  cmp removes bit m.
// Both are pure additions of same-sign terms (exact up to rounding).
//
// The input is split x = x1 x2 (|x1| = n1, |x2| = n2).  Count factorises over
// the split: Count(y, x1 x2) = sum_{y = u1 u2} Count(u1, x1) Count(u2, x2), so
//   pass 1 (columns): for every x2, the n1-symbol sweep over x1 -> F1[c1][x2]
//   pass 2 (rows):    for every code c1, the n2-symbol sweep over x2 -> T[c1][c2]
//   combine:          F_n(y) = sum over splits y = u1 u2 of T[code u1][code u2]
// and the adjoint runs the transposes in reverse order (the combine's
// transpose is a gather fused into the adjoint rows pass).  Each pass keeps
// its whole tile in shared memory; global memory sees each value a few times
// per iteration instead of once per symbol.
#include "bdc_internal.cuh"

#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace {

constexpr int SW_THREADS = 512;

// forward sweep of nn symbols over a tile of (2 << nn) rows x (1 << lw)
// columns held in shared memory (rows >= 2^nn hold the input, rows < 2^nn
// start at zero).  Thread t owns the elements e = t + j*SW_THREADS (j < R) of
// the bottom half for the whole sweep and keeps their values in registers;
// per step it reads the two inserted-bit rows from shared memory, then
// (after a barrier) publishes its new values.  R is a compile-time bound
// on the elements per thread: R * SW_THREADS >= 2^nn << lw.
template <typename T, int R, int NT = SW_THREADS>
__device__ void lsweep_fwd_reg(T *buf, int nn, int lw, int ib = 0) {
    const int tid = threadIdx.x;
    const uint32_t nel = (1u << nn) << lw;
    const uint32_t cmask = (1u << lw) - 1u;
    T own[R];
#pragma unroll
    for (int j = 0; j < R; j++) {
        uint32_t e = tid + j * NT;
        own[j] = (e < nel) ? buf[e] : (T)0;
    }
    for (int i = ib; i < nn; i++) {
        const int m = nn - i - 1;
        const uint32_t row_lo = 1u << m;
        // read phase: other rows' old values from shared memory, own in registers
#pragma unroll
        for (int j = 0; j < R; j++) {
            uint32_t e = tid + j * NT;
            uint32_t P = e >> lw;
            if (e < nel && P >= row_lo) {
                uint32_t c = e & cmask;
                uint32_t i0 = ((P >> m) << (m + 1)) | (P & (row_lo - 1u));
                own[j] = own[j] + buf[(i0 << lw) | c] + buf[((i0 | row_lo) << lw) | c];
            }
        }
        __syncthreads();
        // publish phase
#pragma unroll
        for (int j = 0; j < R; j++) {
            uint32_t e = tid + j * NT;
            if (e < nel && (e >> lw) >= row_lo) buf[e] = own[j];
        }
        __syncthreads();
    }
}

// adjoint sweep: every row Q >= 2^(m+1) adds the row cmp(Q) (bit m removed)
// of the previous level.  Thread t owns e = t + j*NT of the whole
// tile (R * NT >= 2^(nn+1) << lw); afterwards rows [2^nn, 2^(nn+1))
// hold the result.
template <typename T, int R, int NT = SW_THREADS>
__device__ void lsweep_adj_reg(T *buf, int nn, int lw, int ie = 0) {
    const int tid = threadIdx.x;
    const uint32_t nel = (2u << nn) << lw;
    const uint32_t cmask = (1u << lw) - 1u;
    T own[R];
#pragma unroll
    for (int j = 0; j < R; j++) {
        uint32_t e = tid + j * NT;
        own[j] = (e < nel) ? buf[e] : (T)0;
    }
    for (int i = nn - 1; i >= ie; i--) {
        const int m = nn - i - 1;
        const uint32_t row_lo = 2u << m;
        const uint32_t lomask = (1u << m) - 1u;
#pragma unroll
        for (int j = 0; j < R; j++) {
            uint32_t e = tid + j * NT;
            uint32_t Q = e >> lw;
            if (e < nel && Q >= row_lo) {
                uint32_t cq = ((Q >> (m + 1)) << m) | (Q & lomask);
                own[j] += buf[(cq << lw) | (e & cmask)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < R; j++) {
            uint32_t e = tid + j * NT;
            if (e < nel && (e >> lw) >= row_lo) buf[e] = own[j];
        }
        __syncthreads();
    }
}

// dispatch on the tile size (elements per thread rounded up to a power of 2)
// ---------------------------------------------------------------------------
// 4-wide variants: a thread owns groups of 4 consecutive elements (4 columns of
// one row when the tile is at least 4 columns wide, 4 consecutive rows of a
// one-column tile), so one index computation and two 16-byte shared loads
// serve 4 elements.  Same arithmetic, in the same order, as the scalar forms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld4(const float *p, float *v) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double *v) {
    double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ld2(const float *p, float *v) {
    float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ld2(const double *p, double *v) {
    double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x; v[1] = t.y;
}

// forward, tile of >= 4 columns (lw >= 2): group g = 4 columns of row (4g) >> lw
// Final-output hook of the forward sweeps: with a callable `out`, the last
// step's values are handed to out(g, v[4]) (g: the 4-element group) straight
// from registers instead of being published to shared memory.
struct NoOut {};

template <typename T, int G, int NT = SW_THREADS, typename Out = NoOut>
__device__ void lsweep_fwd_cols4(T *buf, int nn, int lw, int ib = 0, Out out = Out()) {
    constexpr bool DIRECT = !std::is_same<Out, NoOut>::value;
    const int tid = threadIdx.x;
    const uint32_t ng = ((1u << nn) << lw) >> 2;
    const uint32_t cmask = (1u << lw) - 1u;
    T own[G][4];
#pragma unroll
    for (int j = 0; j < G; j++) {
        uint32_t g = tid + j * NT;
        if (g < ng) ld4(buf + 4 * g, own[j]);
    }
    for (int i = ib; i < nn; i++) {
        const int m = nn - i - 1;
        const uint32_t row_lo = 1u << m;
        // the 8 lanes of one 16-byte shared-memory phase hold 32/w consecutive
        // rows; when the inserted bit lies inside that span, their i0 rows fall
        // in 4 bank groups twice over.  Lanes 4-7 of each phase then load the
        // i1 row first, which spreads both loads over all 8 bank groups.
        const bool spread = (32u >> lw) > row_lo;
        // group j of a thread: row P0 + j DQ, the same columns; where 2^m
        // divides DQ its inserted-bit rows move by 2 DQ, i.e. 8NT elements
        const uint32_t DQ = (4u * NT) >> lw;
        if (G * NT == (int)ng && (DQ & (row_lo - 1u)) == 0u) {
            const uint32_t P0 = (4u * tid) >> lw, c0 = (4u * tid) & cmask;
            const uint32_t i00 = ((P0 >> m) << (m + 1)) | (P0 & (row_lo - 1u));
            const bool swp = spread && ((tid >> 2) & 1u);
            const T *pa = buf + (((swp ? (i00 | row_lo) : i00) << lw) | c0);
            const T *pb = buf + (((swp ? i00 : (i00 | row_lo)) << lw) | c0);
#pragma unroll
            for (int j = 0; j < G; j++) {
                if (P0 + j * DQ >= row_lo) {
                    T a[4], b[4];
                    ld4(pa + j * 8 * NT, a);
                    ld4(pb + j * 8 * NT, b);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const T r0 = swp ? b[k] : a[k], r1 = swp ? a[k] : b[k];
                        own[j][k] = own[j][k] + r0 + r1;
                    }
                }
            }
        } else
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            uint32_t e = 4 * g, P = e >> lw;
            if (g < ng && P >= row_lo) {
                uint32_t c = e & cmask;
                uint32_t i0 = ((P >> m) << (m + 1)) | (P & (row_lo - 1u));
                const bool swp = spread && ((g >> 2) & 1u);
                T a[4], b[4];
                ld4(buf + (((swp ? (i0 | row_lo) : i0) << lw) | c), a);
                ld4(buf + (((swp ? i0 : (i0 | row_lo)) << lw) | c), b);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const T r0 = swp ? b[k] : a[k], r1 = swp ? a[k] : b[k];
                    own[j][k] = own[j][k] + r0 + r1;
                }
            }
        }
        if (DIRECT && i == nn - 1) break;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            if (g < ng && ((4 * g) >> lw) >= row_lo) st4(buf + 4 * g, own[j]);
        }
        __syncthreads();
    }
    if constexpr (DIRECT) {
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            if (g < ng) out(g, own[j]);
        }
    }
}

// forward, one-column tile (lw == 0): group g = rows 4g..4g+3 (nn >= 2)
template <typename T, int G, int NT = SW_THREADS, typename Out = NoOut>
__device__ void lsweep_fwd_rows4(T *buf, int nn, int ib = 0, Out out = Out()) {
    constexpr bool DIRECT = !std::is_same<Out, NoOut>::value;
    const int tid = threadIdx.x;
    const uint32_t ng = (1u << nn) >> 2;
    T own[G][4];
#pragma unroll
    for (int j = 0; j < G; j++) {
        uint32_t g = tid + j * NT;
        if (g < ng) ld4(buf + 4 * g, own[j]);
    }
    for (int i = ib; i < nn; i++) {
        const int m = nn - i - 1;
        const uint32_t row_lo = 1u << m;
        if (G * NT == (int)ng && m >= 2 && ((4u * NT) & (row_lo - 1u)) == 0u) {
            // group j holds rows 4(tid + j NT) ..: its inserted-bit rows move by
            // 8NT per group (see lsweep_fwd_cols4)
            const uint32_t P00 = 4u * tid;
            const uint32_t i00 = ((P00 >> m) << (m + 1)) | (P00 & (row_lo - 1u));
            const bool swp = ((tid >> 2) & 1u) && row_lo < 32u;
            const T *pa = buf + (swp ? (i00 | row_lo) : i00), *pb = buf + (swp ? i00 : (i00 | row_lo));
#pragma unroll
            for (int j = 0; j < G; j++) {
                if (P00 + j * 4 * NT >= row_lo) {
                    T a[4], b[4];
                    ld4(pa + j * 8 * NT, a);
                    ld4(pb + j * 8 * NT, b);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const T r0 = swp ? b[k] : a[k], r1 = swp ? a[k] : b[k];
                        own[j][k] = own[j][k] + r0 + r1;
                    }
                }
            }
        } else
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            uint32_t P0 = 4 * g;
            if (g < ng && P0 + 3 >= row_lo) {
                T v[8];
                // lanes 4-7 of each 16-byte phase load their second chunk first
                // where the two loads would otherwise meet 4 bank groups twice
                // (inserted bit below position 5); see lsweep_fwd_cols4
                const bool swp = ((g >> 2) & 1u) && row_lo < 32u;
                if (m >= 2) {
                    uint32_t i0 = ((P0 >> m) << (m + 1)) | (P0 & (row_lo - 1u));
                    T a[4], b[4];
                    ld4(buf + (swp ? (i0 | row_lo) : i0), a);
                    ld4(buf + (swp ? i0 : (i0 | row_lo)), b);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const T r0 = swp ? b[k] : a[k], r1 = swp ? a[k] : b[k];
                        own[j][k] = own[j][k] + r0 + r1;
                    }
                } else {
                    // rows 2*P0 .. 2*P0+7 hold both inserted-bit rows of all four
                    T a[4], b[4];
                    ld4(buf + 2 * P0 + (swp ? 4 : 0), a);
                    ld4(buf + 2 * P0 + (swp ? 0 : 4), b);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        v[k] = swp ? b[k] : a[k];
                        v[4 + k] = swp ? a[k] : b[k];
                    }
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (P0 + k < row_lo) continue;
                        // m == 1: i0 = 8g + 4(k>>1) + (k&1), i1 = i0 + 2 ; m == 0: i0 = 8g + 2k, i1 = i0 + 1
                        int i0 = (m == 1) ? (4 * (k >> 1) + (k & 1)) : 2 * k;
                        int i1 = (m == 1) ? i0 + 2 : i0 + 1;
                        own[j][k] = own[j][k] + v[i0] + v[i1];
                    }
                }
            }
        }
        if (DIRECT && i == nn - 1) break;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            uint32_t P0 = 4 * g;
            if (g < ng && P0 + 3 >= row_lo) {
                if (P0 >= row_lo) st4(buf + P0, own[j]);
                else
                    for (int k = 0; k < 4; k++)
                        if (P0 + k >= row_lo) buf[P0 + k] = own[j][k];
            }
        }
        __syncthreads();
    }
    if constexpr (DIRECT) {
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            if (g < ng) out(g, own[j]);
        }
    }
}



// adjoint, tile of >= 4 columns
template <typename T, int G, int NT = SW_THREADS>
__device__ void lsweep_adj_cols4(T *buf, int nn, int lw, int ie = 0) {
    const int tid = threadIdx.x;
    const uint32_t ng = ((2u << nn) << lw) >> 2;
    const uint32_t cmask = (1u << lw) - 1u;
    T own[G][4];
#pragma unroll
    for (int j = 0; j < G; j++) {
        uint32_t g = tid + j * NT;
        if (g < ng) ld4(buf + 4 * g, own[j]);
    }
    // steps m = 0 .. nn-1-ie, two per shared-memory round: with c = cmp_{m+1}(Q),
    // G(m+2 done)[Q] = (G[Q] + G[cmp_m Q]) + (G[c] + G[cmp_m c]), the same
    // additions in the same order as two single steps, half the barriers
    // group j of a thread: row Q0 + j DQ, the same column c.  Where 2^(m+2)
    // divides DQ the partner rows move linearly with j (cmp_m(Q + DQ) =
    // cmp_m(Q) + DQ/2), so their addresses are the first group's plus j times
    // a constant: 2NT elements for cmp_m Q and c, NT for cmp_m c
    const uint32_t DQ = (4u * NT) >> lw;
    const uint32_t Q0 = (4u * tid) >> lw, c0 = (4u * tid) & cmask;
    const int mlast = nn - 1 - ie;
    for (int m = 0; m <= mlast;) {
        const bool two = m + 1 <= mlast;
        const uint32_t row_lo = 2u << m, row_lo2 = 4u << m;
        const uint32_t lomask = (1u << m) - 1u, lomask2 = (2u << m) - 1u;
        if (G * NT == (int)ng && (DQ & (row_lo2 - 1u)) == 0u) {
            const uint32_t cq0 = ((Q0 >> (m + 1)) << m) | (Q0 & lomask);
            const uint32_t c10 = ((Q0 >> (m + 2)) << (m + 1)) | (Q0 & lomask2);
            const uint32_t c1q0 = ((c10 >> (m + 1)) << m) | (c10 & lomask);
            const T *pa = buf + ((cq0 << lw) | c0), *pb = buf + ((c10 << lw) | c0), *pd = buf + ((c1q0 << lw) | c0);
#pragma unroll
            for (int j = 0; j < G; j++) {
                const uint32_t Q = Q0 + j * DQ;
                if (Q >= row_lo) {
                    T a[4];
                    ld4(pa + j * 2 * NT, a);
                    if (two && Q >= row_lo2) {
                        T b[4], d[4];
                        ld4(pb + j * 2 * NT, b);
                        ld4(pd + j * NT, d);
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = (own[j][k] + a[k]) + (b[k] + d[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = own[j][k] + a[k];
                    }
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < G; j++) {
                uint32_t g = tid + j * NT;
                uint32_t e = 4 * g, Q = e >> lw, c = e & cmask;
                if (g < ng && Q >= row_lo) {
                    uint32_t cq = ((Q >> (m + 1)) << m) | (Q & lomask);
                    T a[4];
                    ld4(buf + ((cq << lw) | c), a);
                    if (two && Q >= row_lo2) {
                        uint32_t c1 = ((Q >> (m + 2)) << (m + 1)) | (Q & lomask2);
                        uint32_t c1q = ((c1 >> (m + 1)) << m) | (c1 & lomask);
                        T b[4], d[4];
                        ld4(buf + ((c1 << lw) | c), b);
                        ld4(buf + ((c1q << lw) | c), d);
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = (own[j][k] + a[k]) + (b[k] + d[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = own[j][k] + a[k];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            if (g < ng && ((4 * g) >> lw) >= row_lo) st4(buf + 4 * g, own[j]);
        }
        __syncthreads();
        m += two ? 2 : 1;
    }
}

// adjoint, one-column tile (nn >= 1): group g = rows 4g..4g+3
template <typename T, int G, int NT = SW_THREADS>
__device__ void lsweep_adj_rows4(T *buf, int nn, int ie = 0) {
    const int tid = threadIdx.x;
    const uint32_t ng = (2u << nn) >> 2;
    T own[G][4];
#pragma unroll
    for (int j = 0; j < G; j++) {
        uint32_t g = tid + j * NT;
        if (g < ng) ld4(buf + 4 * g, own[j]);
    }
    // two steps per shared-memory round where possible (see lsweep_adj_cols4);
    // the pairs are (0,1), (2,3), ...
    const int mlast = nn - 1 - ie;
    const bool exact = G * NT == (int)ng;
    for (int m = 0; m <= mlast;) {
        const bool two = m + 1 <= mlast;
        const uint32_t row_lo = 2u << m, row_lo2 = 4u << m;
        const uint32_t lomask = (1u << m) - 1u, lomask2 = (2u << m) - 1u;
        if (exact && m >= 2 && ((4u * NT) & (row_lo2 - 1u)) == 0u) {
            // group j holds rows 4(tid + j NT) ..: partner addresses move by
            // 2NT (cmp_m Q, c) and NT (cmp_m c) per group (see lsweep_adj_cols4)
            const uint32_t Q00 = 4u * tid;
            const uint32_t cq0 = ((Q00 >> (m + 1)) << m) | (Q00 & lomask);
            const uint32_t c10 = ((Q00 >> (m + 2)) << (m + 1)) | (Q00 & lomask2);
            const uint32_t c1q0 = ((c10 >> (m + 1)) << m) | (c10 & lomask);
#pragma unroll
            for (int j = 0; j < G; j++) {
                const uint32_t Q0 = Q00 + j * 4 * NT;
                if (Q0 >= row_lo) {
                    T a[4];
                    ld4(buf + cq0 + j * 2 * NT, a);
                    if (two && Q0 >= row_lo2) {
                        T b[4], d[4];
                        ld4(buf + c10 + j * 2 * NT, b);
                        ld4(buf + c1q0 + j * NT, d);
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = (own[j][k] + a[k]) + (b[k] + d[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = own[j][k] + a[k];
                    }
                }
            }
        } else
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            uint32_t Q0 = 4 * g;
            if (g < ng && Q0 + 3 >= row_lo) {
                if (m >= 2) {
                    uint32_t cq = ((Q0 >> (m + 1)) << m) | (Q0 & lomask);
                    T a[4];
                    ld4(buf + cq, a);
                    if (two && Q0 >= row_lo2) {
                        uint32_t c1 = ((Q0 >> (m + 2)) << (m + 1)) | (Q0 & lomask2);
                        uint32_t c1q = ((c1 >> (m + 1)) << m) | (c1 & lomask);
                        T b[4], d[4];
                        ld4(buf + c1, b);
                        ld4(buf + c1q, d);
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = (own[j][k] + a[k]) + (b[k] + d[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = own[j][k] + a[k];
                    }
                } else if (two) {
                    // m == 0 and 1 together (only when m == 0): row 4g+k gets
                    // (G[4g+k] + G[2g + (k>>1)]) + (G[2g + (k&1)] + G[g]) for g >= 1;
                    // rows 2 and 3 get G[1] (step 0 only)
                    T a[2];
                    ld2(buf + 2 * g, a);
                    if (g >= 1) {
                        const T cg = buf[g];
#pragma unroll
                        for (int k = 0; k < 4; k++) own[j][k] = (own[j][k] + a[k >> 1]) + (a[k & 1] + cg);
                    } else {
                        own[j][2] = own[j][2] + a[1];
                        own[j][3] = own[j][3] + a[1];
                    }
                } else {
                    // m == 1: cmp = 2g, 2g+1, 2g, 2g+1 ; m == 0: cmp = 2g, 2g, 2g+1, 2g+1
                    T a[2];
                    ld2(buf + 2 * g, a);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (Q0 + k < row_lo) continue;
                        own[j][k] = own[j][k] + a[(m == 1) ? (k & 1) : (k >> 1)];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint32_t g = tid + j * NT;
            uint32_t Q0 = 4 * g;
            if (g < ng && Q0 + 3 >= row_lo) {
                if (Q0 >= row_lo) st4(buf + Q0, own[j]);
                else
                    for (int k = 0; k < 4; k++)
                        if (Q0 + k >= row_lo) buf[Q0 + k] = own[j][k];
            }
        }
        __syncthreads();
        m += two ? 2 : 1;
    }
}

// choose the form: R = elements per thread (power of two).  R >= 4 and a tile
// of >= 4 columns or one column use the 4-wide forms; otherwise scalar.
template <typename T, int R, int NT = SW_THREADS, typename Out = NoOut>
__device__ __forceinline__ void lsweep_fwd_any(T *buf, int nn, int lw, int ib = 0, Out out = Out()) {
    if constexpr (R >= 4) {
        if (lw >= 2) { lsweep_fwd_cols4<T, R / 4, NT, Out>(buf, nn, lw, ib, out); return; }
        if (lw == 0 && nn >= 2) { lsweep_fwd_rows4<T, R / 4, NT, Out>(buf, nn, ib, out); return; }
    }
    lsweep_fwd_reg<T, R, NT>(buf, nn, lw, ib);
    if constexpr (!std::is_same<Out, NoOut>::value) {
        // the scalar form publishes; hand the bottom half out from shared memory
        for (uint32_t g = threadIdx.x; g < (((1u << nn) << lw) >> 2); g += NT) {
            T v[4];
            ld4(buf + 4 * g, v);
            out(g, v);
        }
    }
}

template <typename T, int R, int NT = SW_THREADS>
__device__ __forceinline__ void lsweep_adj_any(T *buf, int nn, int lw, int ie = 0) {
    if constexpr (R >= 4) {
        if (lw >= 2) { lsweep_adj_cols4<T, R / 4, NT>(buf, nn, lw, ie); return; }
        if (lw == 0 && nn >= 1) { lsweep_adj_rows4<T, R / 4, NT>(buf, nn, ie); return; }
    }
    lsweep_adj_reg<T, R, NT>(buf, nn, lw, ie);
}

// ---------------------------------------------------------------------------
// Register-resident steps.  Fix the last L input symbols of a tile (its low
// L bits sigma, L = nn - NL).  The first NL forward steps consume the other
// NL symbols and never change the low L bits of a row index: with
// P = (P' << L) | sigma, the insert at position m >= L is the insert at
// m - L on P', and the row ranges map the same way.  So one thread holding
// the 2^NL inputs of its sigma runs those steps in registers, as a sweep
// over a 2^(NL+1)-element tile of its own; likewise the last NL adjoint
// steps.  Only the remaining L steps go through shared memory.
// v[2^NL + r] is the input of row r (r in [0, 2^NL)), rows below start at 0.
// ---------------------------------------------------------------------------
template <typename T, int NL>
__device__ __forceinline__ void local_fwd(T (&v)[2 << NL]) {
#pragma unroll
    for (int P = 0; P < (1 << NL); P++) v[P] = (T)0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        const int m = NL - i - 1;
        // increasing P: every read index is above P, so still the old level
#pragma unroll
        for (int P = 1 << m; P < (1 << NL); P++) {
            const int i0 = ((P >> m) << (m + 1)) | (P & ((1 << m) - 1));
            v[P] = v[P] + v[i0] + v[i0 | (1 << m)];
        }
    }
}

// the last NL adjoint steps; on return v[2^NL + r] holds row r's result
template <typename T, int NL>
__device__ __forceinline__ void local_adj(T (&v)[2 << NL]) {
#pragma unroll
    for (int i = NL - 1; i >= 0; i--) {
        const int m = NL - i - 1;
        // decreasing Q: every read index is below Q, so still the old level
#pragma unroll
        for (int Q = (2 << NL) - 1; Q >= (2 << m); Q--) {
            const int cq = ((Q >> (m + 1)) << m) | (Q & ((1 << m) - 1));
            v[Q] = v[Q] + v[cq];
        }
    }
}

// largest per-thread element count a tile can need (32K FP32 / 16K FP64 elements)
template <typename T>
constexpr int rmax_fwd() { return (sizeof(T) == 4 ? 32768 : 16384) / 2 / SW_THREADS; }
template <typename T>
constexpr int rmax_adj() { return (sizeof(T) == 4 ? 32768 : 16384) / SW_THREADS; }

template <typename T>
__device__ __forceinline__ double block_sum(double v, double *red) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < SW_THREADS / 32; w++) s += red[w];
    return s;
}

// the same reductions in the working precision, sum and maximum together
// (one shared-memory round trip; fixed tree, so deterministic); thread 0
// gets the block's values.  red holds 2 * SW_THREADS / 32 elements.
template <typename T, int NT = SW_THREADS>
__device__ __forceinline__ void block_sum_max_t(T &s, T &m, T *red) {
    const unsigned FULL = 0xffffffffu;
    constexpr int NW = NT / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(FULL, s, o);
        T t = __shfl_xor_sync(FULL, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        red[NW + (threadIdx.x >> 5)] = m;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < NW ? red[threadIdx.x] : (T)0;
        m = threadIdx.x < NW ? red[NW + threadIdx.x] : (T)-INFINITY;
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1) {
            s += __shfl_xor_sync(FULL, s, o);
            T t = __shfl_xor_sync(FULL, m, o);
            m = t > m ? t : m;
        }
    }
}

__device__ __forceinline__ double block_max(double v, double *red) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = -INFINITY;
    if (threadIdx.x == 0)
        for (int w = 0; w < SW_THREADS / 32; w++) s = fmax(s, red[w]);
    return s;
}

// CTAs per SM to plan registers for (512 threads each): as many tiles of
// `bytes` as fit in shared memory, up to `most` (2 CTAs: 64 registers a
// thread, 3: 40).  FP32 only: the FP64 epilogues need more registers.
template <typename T>
constexpr int tile_blocks(size_t bytes, int most) {
    return sizeof(T) != 4 ? 1 : (int)std::min<size_t>((size_t)most, std::max<size_t>(1, (224 * 1024) / bytes));
}

// Complement half mode (p(x) = p(cpl x)): every sweep quantity is invariant
// under complementing all its strings, so only half of it is computed:
//  - column chunks with x2 < 2^(n2-1); the other columns are the complements;
//  - rows c1 in H1 = {empty} u {codes whose first symbol is 0}; row r of the
//    half grid is c1 = 1 (r = 0) or r + 2^(bitlen(r)-1);
//  - output codes in H1, written together with their complement.
__device__ __forceinline__ uint32_t half_row(uint32_t r) { return r == 0 ? 1u : r + (1u << (bitlen32(r) - 1)); }
__device__ __forceinline__ uint32_t cpl_code(uint32_t c) {
    const int j = bitlen32(c) - 1;
    return c ^ ((1u << j) - 1u);
}
__device__ __forceinline__ bool in_h1(uint32_t c) {
    const int j = bitlen32(c) - 1;
    return j == 0 || !((c >> (j - 1)) & 1u);
}

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) and mbarrier, inline PTX (sm_90 and later)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// one 2-D box (x = innermost coordinate, in elements) into shared memory;
// completion is counted in bytes on the mbarrier
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(m))
        : "memory");
}
// bounded wait for phase `parity`: at most `polls` polls (2^22, the
// default, is about a second); false: gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, uint32_t parity, uint32_t polls = (1u << 22)) {
    for (uint32_t it = 0; it < polls; it++)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

struct SweepArgs {
    int n, n1, n2, lw;
    int nblk;                 // column CTAs per instance
    size_t strideN, strideM;  // 2^n, 2^(n+1)
    const double *inst;
    double *part;             // [nd][2][nblk][4]
    int maxblk;
    double q_floor;
    const double *inv_binom;  // [n+1]
    // FP32 copies of the two constants, so FP32 kernels convert nothing
    float q_floor_f;
    float inv_binom_f[BDC_MAXN + 2];
    // column step kernel: load the Gb tile with TMA through the kernel's
    // tensor map (complement half mode, 4 columns, n1 >= 9; see k_cols_adj_l)
    int tma;
    uint32_t tma_polls;       // polls of the TMA tile wait before BDC_ETIMEOUT
};

// rows of the Gb tile that the TMA form loads, in 256-row boxes: slots 0, 1
// are rows [0, 512); for lengths m >= 9, slots 2^(m-9) + 1 + i are the H1
// rows 2^m + 256 i (i < 2^(m-9)).  nslot = 2^(n1-8) + 1.
__device__ __forceinline__ uint32_t tma_slot_row(uint32_t s) {
    if (s < 2u) return 256u * s;
    const uint32_t t = s - 1u;  // in [2^(m-9), 2^(m-8))
    const int m = 9 + (31 - __clz(t));
    return (1u << m) + 256u * (t - (1u << (m - 9)));
}

template <typename T>
__device__ __forceinline__ T inv_binom_t(const SweepArgs &a, int k);
template <>
__device__ __forceinline__ float inv_binom_t<float>(const SweepArgs &a, int k) { return a.inv_binom_f[k]; }
template <>
__device__ __forceinline__ double inv_binom_t<double>(const SweepArgs &a, int k) { return a.inv_binom[k]; }
template <typename T>
__device__ __forceinline__ T q_floor_t(const SweepArgs &a);
template <>
__device__ __forceinline__ float q_floor_t<float>(const SweepArgs &a) { return a.q_floor_f; }
template <>
__device__ __forceinline__ double q_floor_t<double>(const SweepArgs &a) { return a.q_floor; }

// Orbit mean fused into the update (complement half mode).  In half mode
// D(cpl x) = D(x), so the mean of D over the orbit {x, cpl x, rev x, cpl rev x}
// is (D(x) + D(rev x)) / 2, which is symmetric in its two terms: every orbit
// member gets the same bits.  For a column tile (all x1, columns x2 in
// [col0, col0 + w)) the reversed inputs rev(x1 x2) = rev(x2) rev(x1) fill w
// contiguous runs of 2^n1 elements, so they are read coalesced and staged in
// shared memory at the position of x1 = rev(o).  The staged layout XORs the
// top sb bits of x1 into its low bits: the staging writes of one warp then
// hit distinct banks, and each 4-column group stays 16-byte aligned.
__device__ __forceinline__ int swz_bits(int n1, int lw) { return min(max(0, 5 - lw), n1 / 2); }
__device__ __forceinline__ uint32_t swz_pos(uint32_t x1, uint32_t c, int lw, int n1, int sb) {
    return ((x1 << lw) | c) ^ (((x1 >> (n1 - sb)) & ((1u << sb) - 1u)) << lw);
}

template <typename T, int NT = SW_THREADS>
__device__ __forceinline__ void stage_rev_D(T *buf, const T *Dz, int n, int n1, int n2, int lw, uint32_t col0,
                                            int sb) {
    const uint32_t ntop = (1u << n1) << lw, cm = (1u << lw) - 1u;
    const uint32_t full = (1u << n) - 1u;
#pragma unroll 4
    for (uint32_t idx = threadIdx.x; idx < ntop; idx += NT) {
        const uint32_t o = idx >> lw, c = idx & cm;
        uint32_t j = (rev_bits(col0 + c, n2) << n1) | o;
        if ((j >> (n2 - 1)) & 1u) j ^= full;  // held as its complement
        buf[swz_pos(rev_bits(o, n1), c, lw, n1, sb)] = Dz[j];
    }
}

// ---------------------------------------------------------------------------
// pass 1 forward (columns): tile = all x1 x (1<<lw) consecutive x2.
// Prologue applies the pending BA update p <- p 2^{Dbar - shift} and writes
// p back.  With n2 == 0 the pass covers all n symbols and writes q, L.
// ---------------------------------------------------------------------------
template <typename T, int R, bool HALF>
__global__ void __launch_bounds__(SW_THREADS, tile_blocks<T>(2 * R * SW_THREADS * sizeof(T), 2)) k_cols_fwd(SweepArgs a, T *p, const T *D, T *F1, T *q, T *L,
                                                          int apply_update, int mode, int sym_rev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    __shared__ T red[2 * SW_THREADS / 32];
    const int z = blockIdx.y;
    const double *inst = a.inst + z * INST_STRIDE;
    if (!flag_set(inst, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2, lw = a.lw;
    const uint32_t w = 1u << lw;
    const uint32_t col0 = blockIdx.x << lw;
    T *pz = p + z * a.strideN;
    const T *Dz = D + z * a.strideN;
    const bool upd = apply_update && flag_set(inst, I_PENDING);
    const T shift = (T)inst[I_SHIFT];
    const uint32_t ntop = (1u << n1) << lw;
    // orbit mean fused here (half mode, D not yet averaged): the bottom half of
    // the tile holds D(rev x) until each value is used, then is zeroed by its user
    const bool symr = HALF && sym_rev && upd && flag_set(inst, I_SYMNEED);
    const int sb = swz_bits(n1, lw);
    if (symr) {
        stage_rev_D<T>(buf, Dz, a.n, n1, n2, lw, col0, sb);
        __syncthreads();
    }
    T psum = (T)0;  // per-thread partial in the working precision
    if (lw >= 2) {
        // 4 consecutive columns of one row per step: 16-byte global accesses
#pragma unroll 8
        for (uint32_t e = 4 * threadIdx.x; e < ntop; e += 4 * SW_THREADS) {
            uint32_t x1 = e >> lw, c = e & (w - 1u);
            size_t x = ((size_t)x1 << n2) | (col0 + c);
            T v[4], dv[4];
            const T zero[4] = {(T)0, (T)0, (T)0, (T)0};
            ld4(pz + x, v);
            if (upd) {
                ld4(Dz + x, dv);
                if (symr) {
                    T dr[4];
                    const uint32_t sp = swz_pos(x1, c, lw, n1, sb);
                    ld4(buf + sp, dr);
                    st4(buf + sp, zero);
#pragma unroll
                    for (int k = 0; k < 4; k++) dv[k] = (dv[k] + dr[k]) * (T)0.5;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) v[k] = v[k] * exp2_t<T>(dv[k] - shift);
                st4(pz + x, v);
            }
            st4(buf + ntop + e, v);
            if (!symr) st4(buf + e, zero);
            psum += (v[0] + v[1]) + (v[2] + v[3]);
        }
    } else {
        for (uint32_t e = threadIdx.x; e < ntop; e += SW_THREADS) {
            uint32_t x1 = e >> lw, c = e & (w - 1u);
            size_t x = ((size_t)x1 << n2) | (col0 + c);
            T v = pz[x];
            if (upd) {
                T dv = Dz[x];
                if (symr) {
                    const uint32_t sp = swz_pos(x1, c, lw, n1, sb);
                    dv = (dv + buf[sp]) * (T)0.5;
                    buf[sp] = (T)0;
                }
                v = v * exp2_t<T>(dv - shift);
                pz[x] = v;
            }
            buf[ntop + e] = v;
            if (!symr) buf[e] = (T)0;
            psum += v;
        }
    }
    T pmax = (T)0;
    block_sum_max_t<T>(psum, pmax, red);
    if (threadIdx.x == 0 && (mode == MODE_ITER || mode == MODE_DIV)) {
        double *pp = a.part + ((size_t)z * 2 + 0) * a.maxblk * 4 + blockIdx.x * 4;
        // in half mode each column x2 also stands for its complement column
        pp[0] = (double)psum * (HALF ? 2.0 : 1.0);
    }
    __syncthreads();
    lsweep_fwd_any<T, R>(buf, n1, lw);
    if (n2 > 0) {
        T *Fz = F1 + z * a.strideN;
        if (lw >= 2) {
#pragma unroll 8
            for (uint32_t e = w + 4 * threadIdx.x; e < ntop; e += 4 * SW_THREADS) {
                uint32_t row = e >> lw, c = e & (w - 1u);
                T v[4];
                ld4(buf + e, v);
                st4(Fz + (((size_t)row << n2) | (col0 + c)), v);
            }
        } else {
            for (uint32_t e = threadIdx.x + w; e < ntop; e += SW_THREADS) {
                uint32_t row = e >> lw, c = e & (w - 1u);
                Fz[((size_t)row << n2) | (col0 + c)] = buf[e];
            }
        }
    } else {
        T *qz = q + z * a.strideM, *Lz = L + z * a.strideM;
        for (uint32_t c = threadIdx.x + 1; c < (2u << n1); c += SW_THREADS) {
            int k = bitlen32(c) - 1;
            T qv = buf[c] * inv_binom_t<T>(a, k);
            qz[c] = qv;
            Lz[c] = log2_t<T>(mode == MODE_CERT ? fmin(qv, (T)1) : fmax(qv, q_floor_t<T>(a)));
        }
    }
}

// forward rows output: codes c2 < 32 of row c1 go to the transposed Ts, the
// others to Tm row c1 (16-byte stores)
template <typename T, int NT>
__device__ __forceinline__ void store_row_T(const T *buf, T *__restrict__ Tmz, T *__restrict__ Tsz, uint32_t c1, int n1,
                                            int n2) {
    if (threadIdx.x + 1 < min(32u, 1u << n2)) Tsz[((size_t)(threadIdx.x + 1) << (n1 + 1)) + c1] = buf[threadIdx.x + 1];
    T *row = Tmz + ((size_t)c1 << n2);
    for (uint32_t c2 = 32 + 4 * threadIdx.x; c2 < (1u << n2); c2 += 4 * NT) {
        T t4[4];
        ld4(buf + c2, t4);
        st4(row + c2, t4);
    }
}

// pass 2 forward (rows): one row c1 per CTA; input row = F1[c1] (c1 < 2^n1)
// or p[x1 = c1 - 2^n1]; output codes c2 < 32 go to the transposed Ts.
template <typename T, int R, bool HALF>
__global__ void __launch_bounds__(SW_THREADS, tile_blocks<T>(2 * R * SW_THREADS * sizeof(T), R <= 8 ? 3 : 2)) k_rows_fwd(SweepArgs a, const T *p, const T *F1, T *Tm, T *Ts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const int z = blockIdx.y;
    if (!flag_set(a.inst + z * INST_STRIDE, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2;
    const uint32_t c1 = HALF ? half_row(blockIdx.x) : blockIdx.x + 1;
    const uint32_t half = 1u << n2;
    const T *src = (c1 >= (1u << n1)) ? p + z * a.strideN + ((size_t)(c1 - (1u << n1)) << n2)
                                      : F1 + z * a.strideN + ((size_t)c1 << n2);
    if (!HALF) {
#pragma unroll 8
        for (uint32_t e = threadIdx.x; e < half; e += SW_THREADS) {
            buf[half + e] = src[e];
            buf[e] = (T)0;
        }
    } else {
        // columns x2 >= 2^(n2-1) of row c1 are the complement row at column cpl(x2)
        const uint32_t cc = cpl_code(c1), hh = half >> 1, full2 = half - 1u;
        const T *srcm = (cc >= (1u << n1)) ? p + z * a.strideN + ((size_t)(cc - (1u << n1)) << n2)
                                           : F1 + z * a.strideN + ((size_t)cc << n2);
#pragma unroll 8
        for (uint32_t e = threadIdx.x; e < half; e += SW_THREADS) {
            buf[half + e] = (e < hh) ? src[e] : srcm[full2 - e];
            buf[e] = (T)0;
        }
    }
    __syncthreads();
    lsweep_fwd_any<T, R>(buf, n2, 0);
    T *Tmz = Tm + z * a.strideM;
    T *Tsz = Ts + z * ((size_t)32 << (n1 + 1));
    store_row_T<T, SW_THREADS>(buf, Tmz, Tsz, c1, n1, n2);
    (void)half;
}

// combine: F_n(y) = sum over splits of the two passes' outputs; q_k = F_n / C(n,k)
template <typename T, bool HALF>
__global__ void k_combine(SweepArgs a, const T *__restrict__ p, const T *__restrict__ F1, const T *__restrict__ Tm,
                          const T *__restrict__ Ts, T *__restrict__ q, T *__restrict__ L, int mode) {
    const int z = blockIdx.y;
    if (!flag_set(a.inst + z * INST_STRIDE, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2, n = a.n;
    const T *pz = p + z * a.strideN, *Fz = F1 + z * a.strideN, *Tmz = Tm + z * a.strideM;
    const T *Tsz = Ts + z * ((size_t)32 << (n1 + 1));
    T *qz = q + z * a.strideM, *Lz = L + z * a.strideM;
    const uint32_t total = HALF ? (1u << n) : (2u << n);
    const uint32_t hh = 1u << (n2 - 1), full2 = (1u << n2) - 1u;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const uint32_t c = HALF ? half_row(t) : t;
        if (c == 0) continue;
        const int k = bitlen32(c) - 1;
        const uint32_t y = c ^ (1u << k);
        const int jlo = max(0, k - n2), jhi = min(k, n1);
        T acc = (T)0;
        for (int j = jlo; j <= jhi; j++) {
            const int l = k - j;
            uint32_t c1 = (1u << j) | (y >> l);
            uint32_t u2 = y & ((1u << l) - 1u);
            const uint32_t c2 = (1u << l) | u2;
            T v;
            if (l == n2) {
                if (HALF && u2 >= hh) {  // complement column of the complement row
                    c1 = cpl_code(c1);
                    u2 = full2 - u2;
                }
                v = (c1 >= (1u << n1)) ? pz[((size_t)(c1 - (1u << n1)) << n2) | u2] : Fz[((size_t)c1 << n2) | u2];
            } else if (c2 < 32) v = Tsz[((size_t)c2 << (n1 + 1)) + c1];
            else v = Tmz[((size_t)c1 << n2) + c2];
            acc += v;
        }
        T qv = acc * inv_binom_t<T>(a, k);
        T lv = log2_t<T>(mode == MODE_CERT ? fmin(qv, (T)1) : fmax(qv, q_floor_t<T>(a)));
        // a BA iteration needs log2 q only, and in half mode only at the codes
        // the adjoint rows pass gathers: H1 codes, and every code of length <= n2
        const bool keep_q = mode != MODE_ITER;
        if (keep_q) qz[c] = qv;
        Lz[c] = lv;
        if (HALF && k > 0 && (keep_q || k <= n2)) {
            const uint32_t cm = cpl_code(c);
            if (keep_q) qz[cm] = qv;
            Lz[cm] = lv;
        }
    }
}

// The same combine with the codes laid out by length: every CTA holds up to
// CMB_CODES consecutive codes of one length k, so the split range, the source
// array of each split and every shift are uniform across the CTA, and a term
// costs a few integer operations and one load; each of the CMB_THREADS
// threads takes CMB_CODES / CMB_THREADS codes, CMB_THREADS apart.  Codes of
// length k: 2^(k-1) in half mode (those starting with 0), 2^k otherwise.
// Each length below KB has a CTA of its own (a CTA's splits run one after
// another, so these short lengths with their many splits must not queue
// behind each other); longer lengths fill CTAs of CMB_CODES codes.  Measured
// at n = 24 (FP32): 512 codes on 128 threads 47.5 us; 1024 on 256 50 us, 2048
// on 512 53 us, 256 on 64 49 us; two codes a thread (512 on 256, 256 on 128)
// 74-76 us, eight (1024 on 128) 59 us.
constexpr int CMB_LOG = 9, CMB_CODES = 1 << CMB_LOG, CMB_THREADS = 128;
template <typename T, bool HALF>
__global__ void __launch_bounds__(CMB_THREADS) k_combine_k(SweepArgs a, const T *__restrict__ p, const T *__restrict__ F1,
                                                   const T *__restrict__ Tm, const T *__restrict__ Ts,
                                                   T *__restrict__ q, T *__restrict__ L, int mode) {
    constexpr int KB = CMB_LOG + (HALF ? 1 : 0);
    const int z = blockIdx.y;
    // the instance flag is tested only once the first global loads are in
    // flight (the loads before the test read valid memory of any instance)
    const bool active = flag_set(a.inst + z * INST_STRIDE, I_ACTIVE);
    const int n1 = a.n1, n2 = a.n2, n = a.n;
    const T *pz = p + z * a.strideN, *Fz = F1 + z * a.strideN, *Tmz = Tm + z * a.strideM;
    const T *Tsz = Ts + z * ((size_t)32 << (n1 + 1));
    T *qz = q + z * a.strideM, *Lz = L + z * a.strideM;
    const uint32_t hh = 1u << (n2 - 1), full2 = (1u << n2) - 1u;
    const bool keep_q = mode != MODE_ITER;
    // blocks [0, KB): one length k < KB each (at most CMB_CODES codes, all of
    // them, from y = 0); block KB - 1 + b (b >= 1): length KB - 1 + bitlen(b),
    // codes from (b - 2^(k-KB)) CMB_CODES on
    const uint32_t bb = blockIdx.x;
    const bool small = bb < (uint32_t)KB;
    const int k = small ? (int)bb : KB - 1 + bitlen32(bb - KB + 1);
    if (k > n) return;
    {
        const uint32_t cnt = (k == 0) ? 1u : (HALF ? 1u << (k - 1) : 1u << k);
        const uint32_t y0 = small ? 0u : ((bb - KB + 1) - (1u << (k - KB))) << CMB_LOG;
        const int jlo = max(0, k - n2), jhi = min(k, n1);
        // the thread's CMB_CODES / CMB_THREADS codes advance through the splits
        // together: their loads of one split are independent and in flight at once
        constexpr int RC = CMB_CODES / CMB_THREADS;
        T acc[RC];
#pragma unroll
        for (int r = 0; r < RC; r++) acc[r] = (T)0;
#pragma unroll 2
        for (int j = jlo; j <= jhi; j++) {
            const int l = k - j;
            // (a second part of exactly CMB_LOG = n2 symbols spans both of its
            // halves within one CTA, so their complement choice is per code)
            if (!small && l >= CMB_LOG && !(HALF && l == n2 && l == CMB_LOG)) {
                // the CTA's codes share y >> l (y0 is a multiple of 2^CMB_LOG):
                // the term of code y0 + t is src[+-t] for one base per CTA
                const uint32_t u20 = y0 & ((1u << l) - 1u);
                uint32_t c1 = (1u << j) | (y0 >> l);
                const T *src, *arr;
                size_t ext;
                int sgn = 1;
                if (l == n2) {
                    uint32_t u2b = u20;
                    if (HALF && u20 >= hh) {  // complement column of the complement row
                        c1 = c1 ^ ((1u << j) - 1u);
                        u2b = full2 - u20;
                        sgn = -1;
                    }
                    arr = (j == n1) ? pz : Fz;
                    ext = a.strideN;
                    src = ((j == n1) ? pz + ((size_t)(c1 ^ (1u << n1)) << n2) : Fz + ((size_t)c1 << n2)) + u2b;
                } else {
                    arr = Tmz;
                    ext = a.strideM;
                    src = Tmz + ((size_t)c1 << n2) + (1u << l) + u20;
                }
                (void)arr;
                (void)ext;
#pragma unroll
                for (int r = 0; r < RC; r++) {
                    const int off = sgn * (int)(r * CMB_THREADS + threadIdx.x);
                    if (BDC_IN_RANGE((src - arr) + off, ext, a.inst + z * INST_STRIDE)) acc[r] += src[off];
                }
                continue;
            }
#pragma unroll
            for (int r = 0; r < RC; r++) {
                const uint32_t y = y0 + r * CMB_THREADS + threadIdx.x;
                if (y >= cnt) break;
                uint32_t c1 = (1u << j) | (y >> l);
                uint32_t u2 = y & ((1u << l) - 1u);
                T v = (T)0;
                const double *st = a.inst + z * INST_STRIDE;
                (void)st;
                if (l == n2) {
                    if (HALF && u2 >= hh) {  // complement column of the complement row
                        c1 = c1 ^ ((1u << j) - 1u);
                        u2 = full2 - u2;
                    }
                    const size_t ip = ((size_t)(c1 ^ (1u << n1)) << n2) | u2, ifl = ((size_t)c1 << n2) | u2;
                    if (BDC_IN_RANGE(j == n1 ? ip : ifl, a.strideN, st)) v = (j == n1) ? pz[ip] : Fz[ifl];
                } else if (l < 5) {
                    const size_t is = ((size_t)((1u << l) | u2) << (n1 + 1)) + c1;
                    if (BDC_IN_RANGE(is, (size_t)32 << (n1 + 1), st)) v = Tsz[is];
                } else {
                    const size_t im = ((size_t)c1 << n2) + ((1u << l) | u2);
                    if (BDC_IN_RANGE(im, a.strideM, st)) v = Tmz[im];
                }
                acc[r] += v;
            }
        }
        if (!active) return;
#pragma unroll
        for (int r = 0; r < RC; r++) {
            const uint32_t y = y0 + r * CMB_THREADS + threadIdx.x;
            if (y >= cnt) break;
            const T accr = acc[r];
            const uint32_t c = (1u << k) | y;
            T qv = accr * inv_binom_t<T>(a, k);
            T lv = log2_t<T>(mode == MODE_CERT ? fmin(qv, (T)1) : fmax(qv, q_floor_t<T>(a)));
            if (keep_q) qz[c] = qv;
            Lz[c] = lv;
            if (HALF && k > 0 && (keep_q || k <= n2)) {
                const uint32_t cm = c ^ ((1u << k) - 1u);
                if (keep_q) qz[cm] = qv;
                Lz[cm] = lv;
            }
        }
    }
}

// adjoint rows input: buf[c2] = omega_{j+l} L(c1 . u2) for c2 = 2^l + u2
// (l = |u2|, j = |c1|), buf[0] = 0.  For each length l the codes
// (c1 << l) + u2 are 2^l contiguous values: 16-byte loads and stores from l = 2.
template <typename T, int NT>
__device__ __forceinline__ void gather_row_L(T *buf, const T *__restrict__ Lz, const T *__restrict__ om, uint32_t c1,
                                             int j, int n2) {
    if (threadIdx.x < 4) {
        const uint32_t c2 = threadIdx.x;
        T t = (T)0;
        if (c2 > 0) {
            const int l = bitlen32(c2) - 1;
            t = om[j + l] * Lz[(c1 << l) | (c2 ^ (1u << l))];
        }
        buf[c2] = t;
    }
    for (int l = 2; l <= n2; l++) {
        const T wl = om[j + l];
        const T *src = Lz + ((size_t)c1 << l);
        T *dst = buf + (1u << l);
        for (uint32_t t = 4 * threadIdx.x; t < (1u << l); t += 4 * NT) {
            T a4[4];
            ld4(src + t, a4);
#pragma unroll
            for (int k = 0; k < 4; k++) a4[k] = wl * a4[k];
            st4(dst + t, a4);
        }
    }
}

// The same gather as one flat pass (CH * NT * 4 = 2^(n2+1) codes): chunk k
// holds codes 4k .. 4k+3, whose length l and source run follow from the code
// itself, so every thread issues all of its loads before its first store.
template <typename T, int NT, int CH>
__device__ __forceinline__ void gather_row_L_flat(T *buf, const T *__restrict__ Lz, const T *__restrict__ om,
                                                  uint32_t c1, int j) {
    T a4[CH][4];
    T wl[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) {
        const uint32_t code = 4u * (threadIdx.x + i * NT);
        if (code >= 4) {
            const int l = 31 - __clz(code);
            wl[i] = om[j + l];
            ld4(Lz + ((size_t)c1 << l) + (code - (1u << l)), a4[i]);
        } else {
            // codes 1, 2, 3: c1.0 ... (l = 0: the code c1 itself; l = 1: c1 0, c1 1)
            wl[i] = (T)1;
            a4[i][0] = (T)0;
            a4[i][1] = om[j] * Lz[c1];
            a4[i][2] = om[j + 1] * Lz[(size_t)c1 << 1];
            a4[i][3] = om[j + 1] * Lz[((size_t)c1 << 1) | 1u];
        }
    }
#pragma unroll
    for (int i = 0; i < CH; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++) a4[i][k] = wl[i] * a4[i][k];
        st4(buf + 4u * (threadIdx.x + i * NT), a4[i]);
    }
}

// pass 2 adjoint (rows): gather omega_k L(code c1 . c2) over the row, adjoint
// sweep over x2, write the row's top half to Gb[c1][x2].
template <typename T, int R, bool HALF>
__global__ void __launch_bounds__(SW_THREADS, tile_blocks<T>(R * SW_THREADS * sizeof(T), R <= 16 ? 3 : 2)) k_rows_adj(SweepArgs a, const T *Lsrc, const T *omega, T *Gb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const int z = blockIdx.y;
    if (!flag_set(a.inst + z * INST_STRIDE, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2, n = a.n;
    const uint32_t c1 = HALF ? half_row(blockIdx.x) : blockIdx.x + 1;
    const int j = bitlen32(c1) - 1;
    gather_row_L<T, SW_THREADS>(buf, Lsrc + z * a.strideM, omega + z * (n + 1), c1, j, n2);
    __syncthreads();
    lsweep_adj_any<T, R>(buf, n2, 0);
    T *Gz = Gb + z * a.strideM + ((size_t)c1 << n2);
    const uint32_t half = 1u << n2;
#pragma unroll 8
    for (uint32_t e = threadIdx.x; e < half; e += SW_THREADS) Gz[e] = buf[half + e];
    (void)n1;
}

struct EpiArgs {
    const double *hb2;   // [nd][2^n] sum_k rho_k b_k H_k (dual-bound d-gradient)
    const void *Hb;      // [nd][2^n] (T)
    const void *p;       // [nd][2^n] (T)
    void *Dout;          // [nd][2^n] T (MODE_ITER) or double (MODE_DIV / MODE_CERT spare)
    double eH_scale;     // certify: gamma factor on |G|
    double u;            // unit roundoff
};

// pass 1 adjoint (columns): load Gb (or omega L directly when n2 == 0), adjoint
// sweep over x1, then the epilogue D_x = -Hb(x) - G(x) and block partials.
template <typename T, int R, bool HALF>
__global__ void __launch_bounds__(SW_THREADS, tile_blocks<T>(R * SW_THREADS * sizeof(T), 2)) k_cols_adj(SweepArgs a, EpiArgs ep, const T *Gb, const T *Lsrc,
                                                          const T *omega, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    __shared__ double red[SW_THREADS / 32];
    __shared__ T redT[2 * SW_THREADS / 32];
    const int z = blockIdx.y;
    const double *inst = a.inst + z * INST_STRIDE;
    if (!flag_set(inst, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2, lw = a.lw, n = a.n;
    const uint32_t w = 1u << lw;
    const uint32_t col0 = blockIdx.x << lw;
    const uint32_t nall = (2u << n1) << lw;
    if (n2 > 0) {
        const T *Gz = Gb + z * a.strideM;
        const uint32_t full2 = (1u << n2) - 1u;
        if (lw >= 2) {
#pragma unroll 16
            for (uint32_t e = 4 * threadIdx.x; e < nall; e += 4 * SW_THREADS) {
                uint32_t row = e >> lw, c = e & (w - 1u);
                T v[4] = {(T)0, (T)0, (T)0, (T)0};
                if (row) {
                    if (!HALF || in_h1(row)) {
                        ld4(Gz + (((size_t)row << n2) | (col0 + c)), v);
                    } else {
                        // rows outside H1: complement row, complement columns (reversed)
                        T t[4];
                        ld4(Gz + (((size_t)cpl_code(row) << n2) | (full2 - (col0 + c) - 3u)), t);
                        v[0] = t[3]; v[1] = t[2]; v[2] = t[1]; v[3] = t[0];
                    }
                }
                st4(buf + e, v);
            }
        } else if (HALF) {
            for (uint32_t e = threadIdx.x; e < nall; e += SW_THREADS) {
                uint32_t row = e >> lw, c = e & (w - 1u);
                T v = (T)0;
                if (row) v = in_h1(row) ? Gz[((size_t)row << n2) | (col0 + c)]
                                        : Gz[((size_t)cpl_code(row) << n2) | (full2 - (col0 + c))];
                buf[e] = v;
            }
        } else {
            for (uint32_t e = threadIdx.x; e < nall; e += SW_THREADS) {
                uint32_t row = e >> lw, c = e & (w - 1u);
                buf[e] = row ? Gz[((size_t)row << n2) | (col0 + c)] : (T)0;
            }
        }
    } else {
        const T *Lz = Lsrc + z * a.strideM;
        const T *om = omega + z * (n + 1);
        for (uint32_t c = threadIdx.x; c < (2u << n1); c += SW_THREADS)
            buf[c] = c ? om[bitlen32(c) - 1] * Lz[c] : (T)0;
    }
    __syncthreads();
    lsweep_adj_any<T, R>(buf, n1, lw);
    const T *Hbz = reinterpret_cast<const T *>(ep.Hb) + z * a.strideN;
    const T *pz = reinterpret_cast<const T *>(ep.p) + z * a.strideN;
    const uint32_t ntop = (1u << n1) << lw;
    double sZ = 0.0, mD = -INFINITY, sP = 0.0, mP = -INFINITY;
    T tZ = (T)0, tM = (T)-INFINITY;  // MODE_ITER partials in the working precision
    const double add = (mode == MODE_DIV) ? inst[I_SUMP] : 0.0;
    if (mode == MODE_ITER && lw >= 2) {
        T *Dz = reinterpret_cast<T *>(ep.Dout) + z * a.strideN;
#pragma unroll 8
        for (uint32_t e = 4 * threadIdx.x; e < ntop; e += 4 * SW_THREADS) {
            uint32_t x1 = e >> lw, c = e & (w - 1u);
            size_t x = ((size_t)x1 << n2) | (col0 + c);
            T G[4], hb[4], pv[4], Dv[4];
            ld4(buf + ntop + e, G);
            ld4(Hbz + x, hb);
            ld4(pz + x, pv);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                Dv[k] = -hb[k] - G[k];
                tZ += pv[k] * exp2_t<T>(Dv[k]);
                tM = Dv[k] > tM ? Dv[k] : tM;
            }
            st4(Dz + x, Dv);
        }
    }
    for (uint32_t e = threadIdx.x; e < ntop && !(mode == MODE_ITER && lw >= 2); e += SW_THREADS) {
        uint32_t x1 = e >> lw, c = e & (w - 1u);
        size_t x = ((size_t)x1 << n2) | (col0 + c);
        T G = buf[ntop + e];
        T hb = Hbz[x];
        if (mode == MODE_ITER) {
            T Dv = -hb - G;
            reinterpret_cast<T *>(ep.Dout)[z * a.strideN + x] = Dv;
            tZ += pz[x] * exp2_t<T>(Dv);
            tM = Dv > tM ? Dv : tM;
        } else if (mode == MODE_DIV) {
            double Dv = (double)(-hb - G) + add;
            reinterpret_cast<double *>(ep.Dout)[z * a.strideN + x] = Dv;
            mD = fmax(mD, Dv);
        } else if (mode == MODE_DUAL) {
            // q is a full (normalised) output marginal: D = -h(b) - Hb - G
            double Dv = (double)(-hb - G) + inst[I_NEGH];
            reinterpret_cast<double *>(ep.Dout)[z * a.strideN + x] = Dv;
            mD = fmax(mD, Dv);
        } else if (mode == MODE_DUAL_D) {
            double Dv = reinterpret_cast<const double *>(ep.Dout)[z * a.strideN + x];
            double pi = exp2((Dv - inst[I_DUAL_MAXD]) / inst[I_DUAL_TAU]) / inst[I_DUAL_S];
            sZ += pi * (-ep.hb2[z * a.strideN + x] - (double)G);
        } else {  // MODE_CERT (T = double)
            double Gd = (double)G, Hd = (double)hb;
            double Dv = -Hd - Gd;
            double m = __dadd_ru(__dmul_ru(ep.eH_scale, fabs(Gd)),
                                 __dadd_ru(__dmul_ru(1.01 * ep.u, fabs(Hd) + fabs(Gd)), inst[I_EH]));
            double up = __dadd_ru(Dv, m);
            reinterpret_cast<double *>(ep.Dout)[z * a.strideN + x] = Dv;
            double pv = (double)pz[x];
            sZ += pv * exp2(Dv);
            sP += pv;
            mD = fmax(mD, up);
            mP = fmax(mP, Dv);
        }
    }
    if (mode == MODE_ITER) {
        block_sum_max_t<T>(tZ, tM, redT);
        if (threadIdx.x == 0) {
            double *pp = a.part + ((size_t)z * 2 + 1) * a.maxblk * 4 + blockIdx.x * 4;
            pp[0] = (double)tZ * (HALF ? 2.0 : 1.0);  // each column also stands for its complement
            pp[1] = (double)tM;
            pp[2] = 0.0;
            pp[3] = -INFINITY;
        }
        return;
    }
    double s1 = block_sum<T>(sZ, red);
    double s3 = block_sum<T>(sP, red);
    double s2 = block_max(mD, red);
    double s4 = block_max(mP, red);
    if (threadIdx.x == 0) {
        double *pp = a.part + ((size_t)z * 2 + 1) * a.maxblk * 4 + blockIdx.x * 4;
        pp[0] = s1;
        pp[1] = s2;
        pp[2] = s3;
        pp[3] = s4;
    }
}

// ---------------------------------------------------------------------------
// Split-schedule kernels with register-resident steps (BA iterations).  A
// column tile has exactly SW_THREADS << NL inputs, and thread t owns
// c = t mod w and sigma = t / w (the low L = n1 - NL bits of x1): it loads
// its 2^NL inputs x1 = (r << L) | sigma straight into registers, runs the
// first NL steps there, and hands the state to shared memory for the other
// L steps (the adjoint runs the mirror image, and its epilogue reads the
// results from registers).  A row tile (one column, 2^LT threads, L = LT)
// is handled the same way.  Same arithmetic, in the same order, as the
// all-shared-memory kernels.
// ---------------------------------------------------------------------------

template <typename T, int NL, bool HALF, int CT>
__global__ void __launch_bounds__(CT, CT >= 1024 ? 1 : tile_blocks<T>((size_t)CT * (2 << NL) * sizeof(T), 2))
k_cols_fwd_l(SweepArgs a, T *__restrict__ p, const T *__restrict__ D, T *__restrict__ F1, int apply_update,
             int sym_rev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    __shared__ T red[2 * CT / 32];
    constexpr int NI = 1 << NL;
    const int z = blockIdx.y;
    const double *inst = a.inst + z * INST_STRIDE;
    if (!flag_set(inst, I_ACTIVE)) return;
    const int n1 = a.n1, n2 = a.n2, lw = a.lw, L = n1 - NL;
    const uint32_t w = 1u << lw, col0 = blockIdx.x << lw;
    const uint32_t c = threadIdx.x & (w - 1u), sigma = threadIdx.x >> lw;
    T *pz = p + z * a.strideN;
    const T *Dz = D + z * a.strideN;
    const bool upd = apply_update && flag_set(inst, I_PENDING);
    const T shift = (T)inst[I_SHIFT];
    const bool symr = HALF && sym_rev && upd && flag_set(inst, I_SYMNEED);
    const int sb = swz_bits(n1, lw);
    if (symr) {
        stage_rev_D<T, CT>(buf, Dz, a.n, n1, n2, lw, col0, sb);
        __syncthreads();
    }
    // all of a thread's global loads are issued before its first store; input
    // r of this thread sits at x0 + r * xs
    const size_t x0 = ((size_t)sigma << n2) | (col0 + c), xs = (size_t)1 << (L + n2);
    T v[2 * NI];
#pragma unroll
    for (int r = 0; r < NI; r++) v[NI + r] = pz[x0 + r * xs];
    if (upd) {
        // D goes to the bottom half of v, free until the local steps
#pragma unroll
        for (int r = 0; r < NI; r++) v[r] = Dz[x0 + r * xs];
#pragma unroll
        for (int r = 0; r < NI; r++) {
            const uint32_t x1 = ((uint32_t)r << L) | sigma;
            T d = v[r];
            if (symr) d = (d + buf[swz_pos(x1, c, lw, n1, sb)]) * (T)0.5;
            v[NI + r] = v[NI + r] * exp2_t<T>(d - shift);
        }
#pragma unroll
        for (int r = 0; r < NI; r++) pz[x0 + r * xs] = v[NI + r];
    }
    T psum = (T)0;
#pragma unroll
    for (int r = 0; r < NI; r++) psum += v[NI + r];
    if (symr) __syncthreads();  // every staged value is read: the rows are reused below
    local_fwd<T, NL>(v);
#pragma unroll
    // row (r << L) | sigma, column c sits at r * CT + threadIdx.x (2^L w = CT)
#pragma unroll
    for (int r = 1; r < 2 * NI; r++) buf[r * CT + threadIdx.x] = v[r];
    buf[threadIdx.x] = (T)0;  // rows [0, 2^L) start the shared-memory steps at 0
    T pmax = (T)0;
    block_sum_max_t<T, CT>(psum, pmax, red);  // (its barrier also publishes the rows above)
    if (threadIdx.x == 0) {
        double *pp = a.part + ((size_t)z * 2 + 0) * a.maxblk * 4 + blockIdx.x * 4;
        pp[0] = (double)psum * (HALF ? 2.0 : 1.0);  // each column also stands for its complement
    }
    // the last step's values go straight to F1 (rows 1 .. 2^n1 - 1)
    T *Fz = F1 + z * a.strideN;
    lsweep_fwd_any<T, NI, CT>(buf, n1, lw, NL, [&](uint32_t g, const T *v) {
        const uint32_t e = 4 * g, row = e >> lw, cc = e & (w - 1u);
        if (lw >= 2) {
            if (row) st4(Fz + (((size_t)row << n2) | (col0 + cc)), v);
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t ek = e + k, rk = ek >> lw;
                if (rk) Fz[((size_t)rk << n2) | (col0 + (ek & (w - 1u)))] = v[k];
            }
        }
    });
}

// STEP: the iteration boundary in one pass over the tile.  After D and the
// bounds' partial sums of iteration t, the BA update p <- p 2^(D - s) is
// applied in registers (s: the previous iteration's log2 normaliser; p is kept
// unnormalised and its sum is tracked, so any s is exact) and the forward
// columns pass of iteration t+1 runs on the updated inputs, writing F1.  D is
// not stored.
template <typename T, int NL, bool HALF, bool STEP, int CT>
__global__ void __launch_bounds__(CT, CT >= 1024 ? 1 : tile_blocks<T>((size_t)CT * (2 << NL) * sizeof(T), 2))
k_cols_adj_l(SweepArgs a, EpiArgs ep, const T *__restrict__ Gb, T *__restrict__ pw, T *__restrict__ F1,
             int keep_p,  // 0: the updated p is not stored (schedule timing)
             const __grid_constant__ CUtensorMap tmG) {  // Gb as [nd 2^(n1+1) rows][2^n2], used when a.tma
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA form needs a 128-byte aligned tile (its launch adds 128 bytes of
    // dynamic shared memory for this); the dynamic area follows the static one
    T *buf = reinterpret_cast<T *>(smem_raw + (a.tma ? ((0u - smem_u32(smem_raw)) & 127u) : 0u));
    __shared__ T red[2 * CT / 32];
    __shared__ T red2[2 * CT / 32];
    constexpr int NI = 1 << NL;
    const int z = blockIdx.y;
    // the instance flag is tested only once the first global loads are in
    // flight (the loads before the test read valid memory of any instance)
    const bool active = flag_set(a.inst + z * INST_STRIDE, I_ACTIVE);
    const T shift = STEP ? (T)a.inst[z * INST_STRIDE + I_SHIFT] : (T)0;
    const int n1 = a.n1, n2 = a.n2, lw = a.lw, L = n1 - NL;
    const uint32_t w = 1u << lw, col0 = blockIdx.x << lw;
    const uint32_t nall = (2u << n1) << lw;
    const T *Gz = Gb + z * a.strideM;
    const uint32_t full2 = (1u << n2) - 1u;
    bool tma_done = false;
    if constexpr (HALF && STEP && sizeof(T) == 4) {
        // (alignment of the boxes' shared-memory destinations and of the tensor
        // map; anything else keeps the per-thread loads below)
        if (a.tma && (smem_u32(buf) & 127u) == 0 && (reinterpret_cast<uintptr_t>(&tmG) & 63u) == 0) {
            // TMA form (4 columns, n1 >= 9): the H1 rows at this CTA's columns
            // straight into the tile, and at the mirror columns
            // 2^n2 - col0 - 4 .. 2^n2 - col0 - 1 into a staging area after it;
            // each row outside H1 is then its complement row of the staging
            // area with the 4 columns reversed (rows [0, 512) are loaded whole
            // and their rows outside H1 overwritten the same way)
            __shared__ __align__(8) uint64_t mbar;
            T *stage = buf + nall;
            const uint32_t nslot = (1u << (n1 - 8)) + 1u;
            if (threadIdx.x == 0) {
                mbar_init(&mbar, 1);
                mbar_fence_init();
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_expect_tx(&mbar, 2u * nslot * 256u * 4u * (uint32_t)sizeof(T));
                const int y0 = z << (n1 + 1), xm = (int)(full2 - col0 - 3u);
                for (uint32_t sl = 0; sl < nslot; sl++) {
                    const uint32_t row0 = tma_slot_row(sl);
                    tma_load_2d(buf + (row0 << 2), &tmG, (int)col0, y0 + (int)row0, &mbar);
                    tma_load_2d(stage + ((sl * 256u) << 2), &tmG, xm, y0 + (int)row0, &mbar);
                }
            }
            const bool ok = mbar_wait_bounded(&mbar, 0, a.tma_polls);
            if (__syncthreads_or(!ok)) {
                // a copy did not arrive in time: report, wait (bounded) for the
                // copies still in flight into this CTA's shared memory, return
                if (threadIdx.x == 0) {
                    const_cast<double *>(a.inst)[z * INST_STRIDE + I_STATUS] = (double)BDC_ETIMEOUT;
                    (void)mbar_wait_bounded(&mbar, 0);
                }
                __syncthreads();
                return;
            }
            if (!active) return;
            // rows outside H1 (row 0 is zero): k in [2^(j-1), 2^j) is row
            // 2^j | k of length j, complement row 2^j | (2^j - 1 - k)
            for (uint32_t k = threadIdx.x; k < (1u << n1); k += CT) {
                T t4[4] = {(T)0, (T)0, (T)0, (T)0};
                uint32_t r = 0;
                if (k > 0) {
                    const int j = bitlen32(k);
                    r = (1u << j) | k;
                    const uint32_t qo = ((1u << j) - 1u) ^ k, q = (1u << j) | qo;
                    const uint32_t srow = (q < 512u) ? q : (((1u << (j - 9)) + 1u) << 8) + qo;
                    T t[4];
                    ld4(stage + (srow << 2), t);
                    t4[0] = t[3]; t4[1] = t[2]; t4[2] = t[1]; t4[3] = t[0];
                }
                st4(buf + (r << 2), t4);
            }
            tma_done = true;
        }
    }
    if (tma_done) {
    } else if (lw >= 2) {
        // the tile holds 2^(NL+1) CT elements: NI / 2 chunks of 4 per thread,
        // all loaded before the first store
        T t4[NI / 2][4];
#pragma unroll
        for (int i = 0; i < NI / 2; i++) {
            const uint32_t e = 4u * (threadIdx.x + i * CT), row = e >> lw, cc = e & (w - 1u);
#pragma unroll
            for (int k = 0; k < 4; k++) t4[i][k] = (T)0;
            if (row) {
                if (!HALF || in_h1(row)) {
                    ld4(Gz + (((size_t)row << n2) | (col0 + cc)), t4[i]);
                } else {
                    // rows outside H1: complement row, complement columns (reversed)
                    T t[4];
                    ld4(Gz + (((size_t)cpl_code(row) << n2) | (full2 - (col0 + cc) - 3u)), t);
                    t4[i][0] = t[3]; t4[i][1] = t[2]; t4[i][2] = t[1]; t4[i][3] = t[0];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NI / 2; i++) st4(buf + 4u * (threadIdx.x + i * CT), t4[i]);
    } else {
        for (uint32_t e = threadIdx.x; e < nall; e += CT) {
            uint32_t row = e >> lw, cc = e & (w - 1u);
            T t = (T)0;
            if (row) t = (!HALF || in_h1(row)) ? Gz[((size_t)row << n2) | (col0 + cc)]
                                               : Gz[((size_t)cpl_code(row) << n2) | (full2 - (col0 + cc))];
            buf[e] = t;
        }
    }
    if (!active) return;
    __syncthreads();
    lsweep_adj_any<T, 2 * NI, CT>(buf, n1, lw, NL);
    const uint32_t c = threadIdx.x & (w - 1u), sigma = threadIdx.x >> lw;
    T v[2 * NI];
    v[0] = (T)0;
#pragma unroll
    for (int r = 1; r < 2 * NI; r++) v[r] = buf[r * CT + threadIdx.x];  // row (r << L) | sigma, column c
    local_adj<T, NL>(v);
    const T *__restrict__ Hbz = reinterpret_cast<const T *>(ep.Hb) + z * a.strideN;
    // (STEP reads and rewrites p through this one pointer)
    T *__restrict__ pz = (STEP ? pw : const_cast<T *>(reinterpret_cast<const T *>(ep.p))) + z * a.strideN;
    T *__restrict__ Dz = STEP ? nullptr : reinterpret_cast<T *>(ep.Dout) + z * a.strideN;
    // all of a thread's global loads are issued at once, before its first
    // store: Hb into the rows below 2^NL of v (dead after the local steps),
    // p beside it; then D = -Hb - G, and p takes the G rows
    const size_t x0 = ((size_t)sigma << n2) | (col0 + c), xs = (size_t)1 << (L + n2);
    T pv[NI];
#pragma unroll
    for (int r = 0; r < NI; r++) {
        v[r] = Hbz[x0 + r * xs];
        pv[r] = pz[x0 + r * xs];
    }
#pragma unroll
    for (int r = 0; r < NI; r++) {
        v[r] = -v[r] - v[NI + r];
        v[NI + r] = pv[r];
    }
    T tZ = (T)0, tM = (T)-INFINITY;
#pragma unroll
    for (int r = 0; r < NI; r++) {
        const T Dv = v[r];
        tZ += v[NI + r] * exp2_t<T>(Dv);
        tM = Dv > tM ? Dv : tM;
    }
    if constexpr (!STEP) {
#pragma unroll
        for (int r = 0; r < NI; r++) Dz[x0 + r * xs] = v[r];
        block_sum_max_t<T, CT>(tZ, tM, red);
        if (threadIdx.x == 0) {
            double *pp = a.part + ((size_t)z * 2 + 1) * a.maxblk * 4 + blockIdx.x * 4;
            pp[0] = (double)tZ * (HALF ? 2.0 : 1.0);  // each column also stands for its complement
            pp[1] = (double)tM;
            pp[2] = 0.0;
            pp[3] = -INFINITY;
        }
    } else {
        (void)Dz;
        T tP = (T)0;
#pragma unroll
        for (int r = 0; r < NI; r++) tP += v[NI + r];
#pragma unroll
        for (int r = 0; r < NI; r++) v[NI + r] = v[NI + r] * exp2_t<T>(v[r] - shift);
#pragma unroll
        for (int r = 0; r < NI; r++)
            if (keep_p) pz[x0 + r * xs] = v[NI + r];
        block_sum_max_t<T, CT>(tZ, tM, red);
        T unused = (T)0;
        block_sum_max_t<T, CT>(tP, unused, red2);
        if (threadIdx.x == 0) {
            double *pp = a.part + ((size_t)z * 2 + 1) * a.maxblk * 4 + blockIdx.x * 4;
            pp[0] = (double)tZ * (HALF ? 2.0 : 1.0);  // each column also stands for its complement
            pp[1] = (double)tM;
            pp[2] = (double)tP * (HALF ? 2.0 : 1.0);
            pp[3] = -INFINITY;
        }
        // forward columns pass of the next iteration on the updated inputs
        local_fwd<T, NL>(v);
        __syncthreads();  // every thread has read its adjoint rows from buf
#pragma unroll
        for (int r = 1; r < 2 * NI; r++) buf[r * CT + threadIdx.x] = v[r];  // row (r << L) | sigma, column c
        buf[threadIdx.x] = (T)0;  // rows [0, 2^L) start the shared-memory steps at 0
        __syncthreads();
        // the last step's values go straight to F1 (rows 1 .. 2^n1 - 1)
        T *Fz = F1 + z * a.strideN;
        lsweep_fwd_any<T, NI, CT>(buf, n1, lw, NL, [&](uint32_t g, const T *v) {
            const uint32_t e = 4 * g, row = e >> lw, cc = e & (w - 1u);
            if (lw >= 2) {
                if (row) st4(Fz + (((size_t)row << n2) | (col0 + cc)), v);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t ek = e + k, rk = ek >> lw;
                    if (rk) Fz[((size_t)rk << n2) | (col0 + (ek & (w - 1u)))] = v[k];
                }
            }
        });
    }
}

// rows pass, one row c1 per CTA, 2^LT threads, thread = sigma (n2 = NL + LT)
template <typename T, int NL, bool HALF, int LT>
// (register budget for 768 resident threads per SM: 85 registers a thread)
__global__ void __launch_bounds__(1 << LT, LT <= 8 ? 768 / (1 << LT) : 1)
k_rows_fwd_l(SweepArgs a, const T *p, const T *F1, T *Tm, T *Ts) {
    constexpr int ROW_THREADS = 1 << LT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    constexpr int NI = 1 << NL;
    const int z = blockIdx.y;
    // the instance flag is tested only once the first global loads are in
    // flight (the loads before the test read valid memory of any instance)
    const bool active = flag_set(a.inst + z * INST_STRIDE, I_ACTIVE);
    const int n1 = a.n1, n2 = a.n2;  // n2 = NL + LT
    const uint32_t c1 = HALF ? half_row(blockIdx.x) : blockIdx.x + 1;
    const uint32_t half = 1u << n2, sigma = threadIdx.x;
    const T *src = (c1 >= (1u << n1)) ? p + z * a.strideN + ((size_t)(c1 - (1u << n1)) << n2)
                                      : F1 + z * a.strideN + ((size_t)c1 << n2);
    const T *srcm = src;
    if (HALF) {
        // columns x2 >= 2^(n2-1) of row c1 are the complement row at column cpl(x2)
        const uint32_t cc = cpl_code(c1);
        srcm = (cc >= (1u << n1)) ? p + z * a.strideN + ((size_t)(cc - (1u << n1)) << n2)
                                  : F1 + z * a.strideN + ((size_t)cc << n2);
    }
    T v[2 * NI];
#pragma unroll
    for (int r = 0; r < NI; r++) {
        const uint32_t x2 = ((uint32_t)r << LT) | sigma;  // (L == LT)
        v[NI + r] = (HALF && x2 >= (half >> 1)) ? srcm[half - 1u - x2] : src[x2];
    }
    if (!active) return;
    local_fwd<T, NL>(v);
#pragma unroll
    for (int r = 1; r < 2 * NI; r++) buf[(r << LT) | sigma] = v[r];  // (L == LT)
    buf[sigma] = (T)0;
    __syncthreads();
    // the last step's values go straight out: codes c2 < 32 to the transposed
    // Ts, the others to Tm row c1 (16-byte stores)
    T *Tmz = Tm + z * a.strideM;
    T *Tsz = Ts + z * ((size_t)32 << (n1 + 1));
    lsweep_fwd_any<T, NI, ROW_THREADS>(buf, n2, 0, NL, [&](uint32_t g, const T *v) {
        const uint32_t c2 = 4 * g;
        if (c2 >= 32) {
            st4(Tmz + ((size_t)c1 << n2) + c2, v);
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (c2 + k >= 1) Tsz[((size_t)(c2 + k) << (n1 + 1)) + c1] = v[k];
        }
    });
}

template <typename T, int NL, bool HALF, int LT>
__global__ void __launch_bounds__(1 << LT) k_rows_adj_l(SweepArgs a, const T *Lsrc, const T *omega, T *Gb) {
    constexpr int ROW_THREADS = 1 << LT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    constexpr int NI = 1 << NL;
    const int z = blockIdx.y;
    // the instance flag is tested only once the first global loads are in
    // flight (the loads before the test read valid memory of any instance)
    const bool active = flag_set(a.inst + z * INST_STRIDE, I_ACTIVE);
    const int n2 = a.n2, n = a.n;  // n2 = NL + LT
    const uint32_t c1 = HALF ? half_row(blockIdx.x) : blockIdx.x + 1;
    const int j = bitlen32(c1) - 1;
    // (2^(n2+1) codes = NI / 2 chunks of 4 per thread)
    gather_row_L_flat<T, ROW_THREADS, NI / 2>(buf, Lsrc + z * a.strideM, omega + z * (n + 1), c1, j);
    if (!active) return;
    __syncthreads();
    lsweep_adj_any<T, 2 * NI, ROW_THREADS>(buf, n2, 0, NL);
    const uint32_t sigma = threadIdx.x;
    T v[2 * NI];
    v[0] = (T)0;
#pragma unroll
    for (int r = 1; r < 2 * NI; r++) v[r] = buf[(r << LT) | sigma];  // (L == LT)
    local_adj<T, NL>(v);
    T *Gz = Gb + z * a.strideM + ((size_t)c1 << n2);
#pragma unroll
    for (int r = 0; r < NI; r++) Gz[(r << LT) | sigma] = v[NI + r];
}

// cuTensorMapEncodeTiled from the driver (the library links the runtime only)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

// tensor map of an FP32 [nd][2^(n1+1)][2^n2] array seen as rows of 2^n2, box
// 4 columns x 256 rows; false where TMA does not apply or encoding fails
static bool tma_map_rows4(const float *base, int nd, int n1, int n2, CUtensorMap *out) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)1 << n2, (cuuint64_t)nd << (n1 + 1)};
    cuuint64_t strides[1] = {((cuuint64_t)1 << n2) * sizeof(float)};
    cuuint32_t box[2] = {4, 256};
    cuuint32_t es[2] = {1, 1};
    return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// bytes of the TMA form's staging area (the mirror columns' H1 row boxes)
static size_t tma_stage_bytes(int n1) { return (((size_t)1 << (n1 - 8)) + 1) * 256 * 4 * sizeof(float); }

template <typename T>
SweepArgs make_args(bdc_engine *e, PrecBuf<T> &b) {
    SweepArgs a{};
    a.n = e->n;
    a.n1 = b.s.n1;
    a.n2 = b.s.n2;
    a.lw = b.s.lw;
    a.nblk = b.s.nblk_cols;
    a.strideN = (size_t)1 << e->n;
    a.strideM = (size_t)2 << e->n;
    a.inst = e->inst;
    a.part = b.part;
    a.maxblk = part_maxblk(e);
    a.q_floor = e->opt.q_floor;
    a.inv_binom = e->bk + (size_t)4 * e->nd * (e->n + 1);
    a.q_floor_f = (float)e->opt.q_floor;
    a.tma_polls = e->opt.tma_wait_polls == 0 ? (1u << 22)
                                             : (e->opt.tma_wait_polls < 0 ? 0u : (uint32_t)e->opt.tma_wait_polls);
    double c = 1.0;  // C(n,k), exact in double for n <= 28
    for (int k = 0; k <= e->n; k++) {
        a.inv_binom_f[k] = (float)(1.0 / c);
        c = c * (e->n - k) / (k + 1);
    }
    return a;
}

template <typename T>
size_t tile_bytes_cols(const Sched &s) { return ((size_t)2 << s.n1 << s.lw) * sizeof(T); }
template <typename T>
size_t tile_bytes_rows(const Sched &s) { return ((size_t)2 << s.n2) * sizeof(T); }

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// elements per thread of a tile, rounded up to a power of two
inline int r_of(size_t elems) {
    size_t per = (elems + SW_THREADS - 1) / SW_THREADS;
    int r = 1;
    while ((size_t)r < per) r <<= 1;
    return r;
}

// run BODY with the compile-time constant R equal to the runtime value rv
// (rv a power of two in [1, RMAX]); BODY sees `R`.
#define SW_WITH_R(RMAX, rv, BODY)                                                             \
    do {                                                                                      \
        switch (rv) {                                                                         \
            case 1: { constexpr int R = 1; BODY; } break;                                     \
            case 2: { constexpr int R = 2; BODY; } break;                                     \
            case 4: { constexpr int R = 4; BODY; } break;                                     \
            case 8: { constexpr int R = 8; BODY; } break;                                     \
            case 16: { constexpr int R = (16 <= (RMAX) ? 16 : (RMAX)); BODY; } break;         \
            case 32: { constexpr int R = (32 <= (RMAX) ? 32 : (RMAX)); BODY; } break;         \
            default: { constexpr int R = (RMAX); BODY; } break;                               \
        }                                                                                     \
    } while (0)

// run BODY with the compile-time constant NL equal to the runtime value nl
// (3 <= nl <= 5; 5 only for FP32 tiles)
#define SW_WITH_NL(T, nl, BODY)                                                  \
    do {                                                                        \
        switch (nl) {                                                           \
            case 3: { constexpr int NL = 3; BODY; } break;                      \
            case 4: { constexpr int NL = 4; BODY; } break;                      \
            default: { constexpr int NL = (sizeof(T) == 4 ? 5 : 4); BODY; } break; \
        }                                                                       \
    } while (0)

// run BODY with the compile-time constant CT equal to the runtime value ct (512 or 1024)
#define SW_WITH_CT(ct, BODY)                                   \
    do {                                                       \
        if ((ct) == 1024) { constexpr int CT = 1024; BODY; }   \
        else { constexpr int CT = 512; BODY; }                 \
    } while (0)

// run BODY with the compile-time constant LT equal to the runtime value lt (7..9)
#define SW_WITH_LT(lt, BODY)                                \
    do {                                                    \
        switch (lt) {                                       \
            case 7: { constexpr int LT = 7; BODY; } break;  \
            case 8: { constexpr int LT = 8; BODY; } break;  \
            default: { constexpr int LT = 9; BODY; } break; \
        }                                                   \
    } while (0)

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
Sched make_sched(int n, int elem_bytes, int n2_override, int w_override) {
    Sched s{};
    const int tile = (elem_bytes == 4) ? 32768 : 16384;  // elements per CTA tile (128 KB)
    int nsingle = 0;
    while ((2 << (nsingle + 1)) <= tile) nsingle++;       // 2^(n+1) <= tile
    // the streaming schedule: asked for (n2_override < 0), or no split of n
    // into column and row tiles of at most `tile` elements exists (n > 2 nsingle)
    if (n2_override < 0 || (n > 2 * nsingle && n2_override == 0)) {
        s.n1 = n;
        s.n2 = -1;
        s.lw = 0;
        s.nblk_cols = 1024;  // CTAs of the streaming epilogues (block partials per instance)
        return s;
    }
    if (n <= nsingle && n2_override == 0) {
        s.n1 = n;
        s.n2 = 0;
        s.lw = 0;
        s.nblk_cols = 1;
        return s;
    }
    // rows pass: 2^(n2+1) elements per CTA; 16K keeps the FP32 rows tile at
    // 64 KB (several CTAs per SM) and every thread's elements in registers
    int n2max = 13;
    int n2 = n2_override ? n2_override : std::min(n - 1, n2max);
    if (n2 < 5) n2 = std::min(5, n - 1);
    if (n - n2 > nsingle) n2 = n - nsingle;  // the columns tile must hold 2^(n1+1) rows
    if (((size_t)2 << n2) > (size_t)tile) {   // nor can a row tile hold 2^(n2+1): stream
        s.n1 = n;
        s.n2 = -1;
        s.lw = 0;
        s.nblk_cols = 1024;
        return s;
    }
    s.n2 = n2;
    s.n1 = n - n2;
    int lw = 0;
    while (lw < 5 && lw < n2 && ((size_t)2 << s.n1 << (lw + 1)) <= (size_t)tile) lw++;
    if (w_override) {
        lw = 0;
        while ((1 << (lw + 1)) <= w_override) lw++;
        // clamp to a tile that fits and to at most the 2^n2 columns
        while (lw > 0 && (((size_t)2 << s.n1 << lw) > (size_t)tile || lw > n2)) lw--;
    }
    s.lw = lw;
    s.nblk_cols = 1 << (n2 - lw);
    return s;
}

template <typename T>
cudaError_t prepare_all(size_t cols_bytes, size_t rows_bytes) {
    cudaError_t err = cudaSuccess;
#define PREP_ONE_H(RR, H)                                                                                        \
    if (RR <= rmax_fwd<T>()) {                                                                                   \
        if (err == cudaSuccess) err = allow_smem(k_cols_fwd<T, (RR <= rmax_fwd<T>() ? RR : 1), H>, cols_bytes); \
        if (err == cudaSuccess) err = allow_smem(k_rows_fwd<T, (RR <= rmax_fwd<T>() ? RR : 1), H>, rows_bytes); \
    }                                                                                                            \
    if (RR <= rmax_adj<T>()) {                                                                                   \
        if (err == cudaSuccess) err = allow_smem(k_cols_adj<T, (RR <= rmax_adj<T>() ? RR : 1), H>, cols_bytes); \
        if (err == cudaSuccess) err = allow_smem(k_rows_adj<T, (RR <= rmax_adj<T>() ? RR : 1), H>, rows_bytes); \
    }
#define PREP_ONE(RR) PREP_ONE_H(RR, false) PREP_ONE_H(RR, true)
    PREP_ONE(1) PREP_ONE(2) PREP_ONE(4) PREP_ONE(8) PREP_ONE(16) PREP_ONE(32) PREP_ONE(64)
#define PREP_L(NL, H)                                                                        \
    if (err == cudaSuccess) err = allow_smem(k_cols_fwd_l<T, NL, H, 512>, cols_bytes);       \
    if (err == cudaSuccess) err = allow_smem(k_cols_fwd_l<T, NL, H, 1024>, cols_bytes);      \
    if (err == cudaSuccess) err = allow_smem(k_cols_adj_l<T, NL, H, false, 512>, cols_bytes); \
    if (err == cudaSuccess) err = allow_smem(k_cols_adj_l<T, NL, H, true, 512>, cols_bytes);  \
    if (err == cudaSuccess) err = allow_smem(k_cols_adj_l<T, NL, H, false, 1024>, cols_bytes); \
    if (err == cudaSuccess) err = allow_smem(k_cols_adj_l<T, NL, H, true, 1024>, cols_bytes);  \
    if (err == cudaSuccess) err = allow_smem(k_rows_adj_l<T, NL, H, 9>, rows_bytes);
    PREP_L(3, false) PREP_L(3, true) PREP_L(4, false) PREP_L(4, true)
    if constexpr (sizeof(T) == 4) { PREP_L(5, false) PREP_L(5, true) }
#undef PREP_L
    constexpr int NLR = sizeof(T) == 4 ? 5 : 4;
#define PREP_R(LT, H) \
    if (err == cudaSuccess) err = allow_smem(k_rows_fwd_l<T, NLR, H, LT>, rows_bytes);
    PREP_R(7, false) PREP_R(7, true) PREP_R(8, false) PREP_R(8, true) PREP_R(9, false) PREP_R(9, true)
#undef PREP_R
#undef PREP_ONE
#undef PREP_ONE_H
    return err;
}

template <typename T>
bdc_status sweep_prepare(bdc_engine *e, PrecBuf<T> &b) {
    const size_t big = (size_t)(sizeof(T) == 4 ? 32768 : 16384) * sizeof(T);
    BDC_CUDA_TRY(prepare_all<T>(big, big));
    (void)e;
    (void)b;
    return BDC_OK;
}

bool half_possible(const Sched &s) { return s.n2 > 0 && s.lw < s.n2 && s.n1 >= 1; }

// register-resident steps (bits of opt.use_regsteps: 1 forward rows,
// 2 adjoint rows, 4 forward columns, 8 adjoint columns): NL of a tile, 0
// where they are off or do not apply.  A column tile must hold
// SW_THREADS << NL inputs; a forward row tile runs NL = 5 (FP32) / 4 (FP64)
// on 2^(n2 - NL) threads, an adjoint row tile NL = n2 - 9 on 512 threads.
// threads of a register-step column CTA: 1024 where one tile fills an SM's
// shared memory (one CTA per SM), else 512 (two CTAs per SM)
template <typename T>
static int ct_cols(const Sched &s) { return tile_bytes_cols<T>(s) > 112 * 1024 ? 1024 : 512; }
template <typename T>
static int nl_cols(const bdc_engine *e, const Sched &s, int bit) {
    const int nl = s.n1 + s.lw - (ct_cols<T>(s) == 1024 ? 10 : 9), nmax = sizeof(T) == 4 ? 5 : 4;
    return ((e->opt.use_regsteps & bit) && s.n2 > 0 && nl >= 3 && nl <= nmax && nl <= s.n1) ? nl : 0;
}
template <typename T>
static int nl_rows_fwd(const bdc_engine *e, const Sched &s) {
    const int nl = sizeof(T) == 4 ? 5 : 4, lt = s.n2 - nl;
    return ((e->opt.use_regsteps & 1) && s.n2 > 0 && lt >= 7 && lt <= 9) ? nl : 0;
}
template <typename T>
static int nl_rows_adj(const bdc_engine *e, const Sched &s) {
    const int nl = s.n2 - 9, nmax = sizeof(T) == 4 ? 5 : 4;
    return ((e->opt.use_regsteps & 2) && s.n2 > 0 && nl >= 3 && nl <= nmax) ? nl : 0;
}

template <typename T>
bool step_possible(const bdc_engine *e, const Sched &s) {
    return e->opt.fuse_update && nl_cols<T>(e, s, 4) && nl_cols<T>(e, s, 8);
}

template <typename T>
bdc_status sweep_forward(bdc_engine *e, PrecBuf<T> &b, const T *p_src, int apply_update, int mode, bool half,
                         bool sym_rev, bool cols, bool rest) {
    if (b.s.n2 < 0) return stream_forward<T>(e, b, p_src, apply_update, mode);
    SweepArgs a = make_args(e, b);
    const Sched &s = b.s;
    half = half && half_possible(s);
    size_t sm1 = tile_bytes_cols<T>(s);
    T *p = const_cast<T *>(p_src);
    dim3 g1(half ? s.nblk_cols / 2 : s.nblk_cols, e->nd);
    const int rc = r_of(((size_t)1 << s.n1) << s.lw);
    const int nlc = (mode == MODE_ITER) ? nl_cols<T>(e, s, 4) : 0;
    const int ct = ct_cols<T>(s);
    if (!cols && s.n2 > 0) {
        // F1 is current (written by the previous stepped adjoint pass)
    } else if (nlc && half)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_fwd_l<T, NL, true, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, p, b.D, b.F1, apply_update, sym_rev ? 1 : 0))));
    else if (nlc)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_fwd_l<T, NL, false, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, p, b.D, b.F1, apply_update, 0))));
    else if (half)
        SW_WITH_R(rmax_fwd<T>(), rc, (k_cols_fwd<T, R, true><<<g1, SW_THREADS, sm1, e->stream>>>(
                                         a, p, b.D, b.F1, b.q, b.L, apply_update, mode, sym_rev ? 1 : 0)));
    else
        SW_WITH_R(rmax_fwd<T>(), rc, (k_cols_fwd<T, R, false><<<g1, SW_THREADS, sm1, e->stream>>>(
                                         a, p, b.D, b.F1, b.q, b.L, apply_update, mode, 0)));
    if (cols || s.n2 == 0) {
        e->launches++; stage_mark(e, "cols_fwd");
        BDC_CUDA_TRY(cudaGetLastError());
        e->f1_current[sizeof(T) == 4 ? 0 : 1] = false;  // F1 now holds this pass's p_src / mode
    }
    if (!rest) return BDC_OK;
    if (s.n2 > 0) {
        size_t sm2 = tile_bytes_rows<T>(s);
        dim3 g2(half ? (1u << s.n1) : (2u << s.n1) - 1u, e->nd);
        const int rr = r_of((size_t)1 << s.n2);
        const int nlr = nl_rows_fwd<T>(e, s);
        constexpr int NLR = sizeof(T) == 4 ? 5 : 4;
        if (nlr && half)
            SW_WITH_LT(s.n2 - nlr, (k_rows_fwd_l<T, NLR, true, LT><<<g2, 1 << LT, sm2, e->stream>>>(a, p, b.F1, b.Tm, b.Ts)));
        else if (nlr)
            SW_WITH_LT(s.n2 - nlr, (k_rows_fwd_l<T, NLR, false, LT><<<g2, 1 << LT, sm2, e->stream>>>(a, p, b.F1, b.Tm, b.Ts)));
        else if (half)
            SW_WITH_R(rmax_fwd<T>(), rr,
                      (k_rows_fwd<T, R, true><<<g2, SW_THREADS, sm2, e->stream>>>(a, p, b.F1, b.Tm, b.Ts)));
        else
            SW_WITH_R(rmax_fwd<T>(), rr,
                      (k_rows_fwd<T, R, false><<<g2, SW_THREADS, sm2, e->stream>>>(a, p, b.F1, b.Tm, b.Ts)));
        e->launches++; stage_mark(e, "rows_fwd");
        BDC_CUDA_TRY(cudaGetLastError());
        // blocks of CMB_CODES codes of one length (k_combine_k)
        const int kb = CMB_LOG + (half ? 1 : 0);
        dim3 g3(e->n >= kb ? (1u << (e->n - kb + 1)) - 1u + kb : (unsigned)e->n + 1u, e->nd);
        if (half) k_combine_k<T, true><<<g3, CMB_THREADS, 0, e->stream>>>(a, p, b.F1, b.Tm, b.Ts, b.q, b.L, mode);
        else k_combine_k<T, false><<<g3, CMB_THREADS, 0, e->stream>>>(a, p, b.F1, b.Tm, b.Ts, b.q, b.L, mode);
        e->launches++; stage_mark(e, "combine");
        BDC_CUDA_TRY(cudaGetLastError());
    }
    return BDC_OK;
}

template <typename T>
bdc_status sweep_adjoint(bdc_engine *e, PrecBuf<T> &b, const T *Lsrc, const T *omega, T *Dout, int mode, bool half,
                         bool step, bool keep_p) {
    if (b.s.n2 < 0) return stream_adjoint<T>(e, b, Lsrc, omega, Dout, mode);
    SweepArgs a = make_args(e, b);
    const Sched &s = b.s;
    half = half && half_possible(s);
    if (s.n2 > 0) {
        size_t sm2 = tile_bytes_rows<T>(s);
        dim3 g2(half ? (1u << s.n1) : (2u << s.n1) - 1u, e->nd);
        const int rr = r_of((size_t)2 << s.n2);
        const int nlr = nl_rows_adj<T>(e, s);
        if (nlr && half)
            SW_WITH_NL(T, nlr, (k_rows_adj_l<T, NL, true, 9><<<g2, SW_THREADS, sm2, e->stream>>>(a, Lsrc, omega, b.Gb)));
        else if (nlr)
            SW_WITH_NL(T, nlr, (k_rows_adj_l<T, NL, false, 9><<<g2, SW_THREADS, sm2, e->stream>>>(a, Lsrc, omega, b.Gb)));
        else if (half)
            SW_WITH_R(rmax_adj<T>(), rr,
                      (k_rows_adj<T, R, true><<<g2, SW_THREADS, sm2, e->stream>>>(a, Lsrc, omega, b.Gb)));
        else
            SW_WITH_R(rmax_adj<T>(), rr,
                      (k_rows_adj<T, R, false><<<g2, SW_THREADS, sm2, e->stream>>>(a, Lsrc, omega, b.Gb)));
        e->launches++; stage_mark(e, "rows_adj");
        BDC_CUDA_TRY(cudaGetLastError());
    }
    EpiArgs ep{};
    ep.hb2 = e->pcert;
    ep.Hb = b.Hb;
    ep.p = (mode == MODE_CERT) ? (const void *)e->pcert : (const void *)b.p;
    ep.Dout = Dout;
    ep.u = 1.1102230246251565e-16;
    {
        // gamma_{n+8} * 1.01 + 1.01 u
        double m = e->n + 8;
        ep.eH_scale = 1.01 * (m * ep.u / (1.0 - m * ep.u)) + 1.01 * ep.u;
    }
    size_t sm1 = tile_bytes_cols<T>(s);
    dim3 g1(half ? s.nblk_cols / 2 : s.nblk_cols, e->nd);
    const int rc = r_of(((size_t)2 << s.n1) << s.lw);
    const int nlc = (mode == MODE_ITER) ? nl_cols<T>(e, s, 8) : 0;
    const int ct = ct_cols<T>(s);
    CUtensorMap tmG;
    memset(&tmG, 0, sizeof(tmG));
    a.tma = 0;
    if (sizeof(T) == 4 && step && nlc && half && e->opt.use_tma && s.lw == 2 && s.n1 >= 9 && ct == 512 &&
        tma_map_rows4(reinterpret_cast<const float *>(b.Gb), e->nd, s.n1, s.n2, &tmG)) {
        a.tma = 1;
        sm1 += tma_stage_bytes(s.n1) + 128;
    }
    if (step && nlc && half)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_adj_l<T, NL, true, true, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, ep, b.Gb, b.p, b.F1, keep_p ? 1 : 0, tmG))));
    else if (step && nlc)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_adj_l<T, NL, false, true, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, ep, b.Gb, b.p, b.F1, keep_p ? 1 : 0, tmG))));
    else if (nlc && half)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_adj_l<T, NL, true, false, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, ep, b.Gb, nullptr, nullptr, 1, tmG))));
    else if (nlc)
        SW_WITH_CT(ct, SW_WITH_NL(T, nlc, (k_cols_adj_l<T, NL, false, false, CT><<<g1, CT, sm1, e->stream>>>(
                                              a, ep, b.Gb, nullptr, nullptr, 1, tmG))));
    else if (half)
        SW_WITH_R(rmax_adj<T>(), rc,
                  (k_cols_adj<T, R, true><<<g1, SW_THREADS, sm1, e->stream>>>(a, ep, b.Gb, Lsrc, omega, mode)));
    else
        SW_WITH_R(rmax_adj<T>(), rc,
                  (k_cols_adj<T, R, false><<<g1, SW_THREADS, sm1, e->stream>>>(a, ep, b.Gb, Lsrc, omega, mode)));
    e->launches++; stage_mark(e, (step && nlc) ? "cols_step" : "cols_adj");
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}

template bdc_status sweep_prepare<float>(bdc_engine *, PrecBuf<float> &);
template bdc_status sweep_prepare<double>(bdc_engine *, PrecBuf<double> &);
template bdc_status sweep_forward<float>(bdc_engine *, PrecBuf<float> &, const float *, int, int, bool, bool, bool,
                                         bool);
template bdc_status sweep_forward<double>(bdc_engine *, PrecBuf<double> &, const double *, int, int, bool, bool, bool,
                                          bool);
template bdc_status sweep_adjoint<float>(bdc_engine *, PrecBuf<float> &, const float *, const float *, float *, int, bool,
                                         bool, bool);
template bdc_status sweep_adjoint<double>(bdc_engine *, PrecBuf<double> &, const double *, const double *, double *, int,
                                          bool, bool, bool);
template bool step_possible<float>(const bdc_engine *, const Sched &);
template bool step_possible<double>(const bdc_engine *, const Sched &);

// ---------------------------------------------------------------------------
// Output marginal without any device allocation.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// CUDA graph being captured by someone else, plugins whose host framework
// owns every allocation and forbids cudaMalloc, or memory-accounted jobs
// that must not grow the device heap.  For them, the forward sweep below
// keeps all of its scratch (the column-pass output, the row-pass output, the
// log table and a few scalars) in one file-scope device array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it
// until the process exits.  The caller passes only the input distribution
// and the output buffer.
//
// Limits and sharing: n <= BDC_STATIC_MAXN (the array is sized for it); all
// calls on a device share the one array and it keeps the last call's values,
// so calls that overlap on the GPU (different streams, or the same stream
// from two host threads without ordering) race and must be serialised by the
// caller.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and sets the kernels'
// shared-memory limits; make that first call before any stream capture.
// ---------------------------------------------------------------------------
namespace {

constexpr int STATIC_MAXN = 18;
// scalars and weights (256) + F1 (2^n) + Tm (2^(n+1)) + Ts (32 * 2^(n1+1), n1 <= 5 with the FP64
// schedule for n <= 18) + L (2^(n+1)): 1,313,024 doubles = 10.5 MB
constexpr size_t STATIC_DOUBLES = 256 + ((size_t)5 << STATIC_MAXN) + (size_t)32 * 64;

static __device__ __align__(256) double g_static_scratch[STATIC_DOUBLES];

__global__ void k_static_init(int n, double d, double *inst, double *wk, double *q_out) {
    int t = threadIdx.x;
    if (t < INST_STRIDE) inst[t] = (t == I_ACTIVE) ? 1.0 : 0.0;
    if (t <= n) wk[t] = pow(d, (double)(n - t)) * pow(1.0 - d, (double)t);  // d^(n-k) (1-d)^k
    if (t == 0) q_out[0] = 0.0;
}

// Per-device set-up state.  The set-up runs under a mutex so that two host
// threads making a device's first call at the same time do it once; later
// calls read the published address without taking the lock.
struct StaticDev {
    std::atomic<double *> base{nullptr};
    int sms = 0;  // multiprocessor count of the device (grid cap of the combine)
};
StaticDev g_static_dev[64];
std::mutex g_static_mu;

}  // namespace

extern "C" bdc_status bdc_output_marginal_static(int n, double d, const double *p_dev, double *q_dev,
                                                 void *cuda_stream) {
    if (n < 1 || n > STATIC_MAXN) {
        bdc_set_error("bdc_output_marginal_static: n must be in [1, 18]; the fixed scratch array holds no more");
        return BDC_EINVAL;
    }
    if (!(d >= 0.0 && d <= 1.0) || !p_dev || !q_dev) {
        bdc_set_error("bdc_output_marginal_static: need 0 <= d <= 1 and non-NULL p, q");
        return BDC_EINVAL;
    }
    int dev = 0;
    BDC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        bdc_set_error("bdc_output_marginal_static: device index above 63");
        return BDC_EINVAL;
    }
    const Sched s = make_sched(n, 8, 0, 0);
    if (!g_static_dev[dev].base.load(std::memory_order_acquire)) {
        // once per device, with that device current
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_dev[dev].base.load(std::memory_order_relaxed)) {
            void *ptr = nullptr;
            cudaError_t err = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (err != cudaSuccess || !ptr) {
                bdc_set_error(std::string("bdc_output_marginal_static: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(err));
                return BDC_ECUDA;
            }
            int sms = 0;
            BDC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            const size_t big = (size_t)16384 * sizeof(double);
            BDC_CUDA_TRY(prepare_all<double>(big, big));
            g_static_dev[dev].sms = std::max(1, sms);
            g_static_dev[dev].base.store((double *)ptr, std::memory_order_release);
        }
    }
    double *base = g_static_dev[dev].base.load(std::memory_order_acquire);
    const int sms = g_static_dev[dev].sms;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t N = (size_t)1 << n;
    double *inst = base;                       // INST_STRIDE doubles
    double *wk = base + 64;                    // n+1 doubles
    double *F1 = base + 256;                   // 2^n
    double *Tm = F1 + N;                       // 2^(n+1)
    double *Ts = Tm + 2 * N;                   // 32 * 2^(n1+1)
    double *L = Ts + (size_t)32 * ((size_t)2 << s.n1);  // 2^(n+1)
    double *part = base;                       // block partials: not written in this mode
    if ((size_t)(L + 2 * N - base) > STATIC_DOUBLES) {
        bdc_set_error("bdc_output_marginal_static: schedule does not fit the fixed scratch array");
        return BDC_EINVAL;
    }
    SweepArgs a{};
    a.n = n;
    a.n1 = s.n1;
    a.n2 = s.n2;
    a.lw = s.lw;
    a.nblk = s.nblk_cols;
    a.strideN = N;
    a.strideM = 2 * N;
    a.inst = inst;
    a.part = part;
    a.maxblk = 0;
    a.q_floor = 1e-300;
    a.inv_binom = wk;  // the combine's per-length weight: d^(n-k)(1-d)^k gives q(y) = sum_x p W
    k_static_init<<<1, 64, 0, st>>>(n, d, inst, wk, q_dev);
    double *p = const_cast<double *>(p_dev);  // read only: no update is applied
    const int rc = r_of(((size_t)1 << s.n1) << s.lw);
    SW_WITH_R(rmax_fwd<double>(), rc,
              (k_cols_fwd<double, R, false><<<dim3(s.nblk_cols, 1), SW_THREADS, tile_bytes_cols<double>(s), st>>>(
                  a, p, p, F1, q_dev, L, 0, MODE_DUAL, 0)));
    if (s.n2 > 0) {
        const int rr = r_of((size_t)1 << s.n2);
        SW_WITH_R(rmax_fwd<double>(), rr,
                  (k_rows_fwd<double, R, false><<<dim3((2u << s.n1) - 1u, 1), SW_THREADS, tile_bytes_rows<double>(s), st>>>(
                      a, p, F1, Tm, Ts)));
        int nb = (int)std::min<size_t>((2 * N) / 256 + 1, (size_t)sms * 16);
        k_combine<double, false><<<dim3(nb, 1), 256, 0, st>>>(a, p, F1, Tm, Ts, q_dev, L, MODE_DUAL);
    }
    BDC_CUDA_TRY(cudaGetLastError());
    return BDC_OK;
}
