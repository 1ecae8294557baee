// Microbenchmarks of the device peaks the sweep and walk kernels are measured
// against, run in the same process as the measurement they serve: FP32 and
// FP64 add/FMA issue rates (the sweeps are chains of additions, one pipe
// slot each), L2 read bandwidth on a buffer that stays resident in L2, and
// shared-memory bandwidth (16-byte accesses).  Every kernel is plain CUDA,
// timed with CUDA events on the caller's stream after a warm-up launch.
#include "bdc_internal.cuh"

#include <algorithm>

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;    // independent dependency chains per thread
constexpr int PK_ITERS = 4096;  // FMAs per chain

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_rate(T seed, T *sink) {
    T a[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, s = (T)1e-7;
#pragma unroll 16
    for (int i = 0; i < PK_ITERS; i++)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; c++) a[c] = a[c] * m + s;
    T t = (T)0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) t += a[c];
    if (t == (T)-1) sink[threadIdx.x] = t;  // never true: keeps the chains live
}

// the grid reads the `words` 16-byte words of buf `reps` times over
// (L2-resident after the first pass: the buffer is far below the L2 size)
__global__ void __launch_bounds__(PK_THREADS) k_l2_read(const uint4 *__restrict__ buf, size_t words, int reps,
                                                        unsigned *sink) {
    unsigned acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; r++) {
        // each pass starts at a different offset so CTAs do not march in step
        const size_t off = ((size_t)blockIdx.x * 977 + (size_t)r * 131071) % words;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
            size_t j = i + off;
            if (j >= words) j -= words;
            const uint4 v = __ldcg(buf + j);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

// shared memory: 16-byte loads from a 32 KB tile, conflict-free (a warp's
// 32 loads cover 512 consecutive bytes)
__global__ void __launch_bounds__(PK_THREADS) k_smem_rate(int reps, unsigned *sink) {
    __shared__ uint4 tile[2048];
    for (int i = threadIdx.x; i < 2048; i += PK_THREADS) tile[i] = make_uint4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    uint4 acc = make_uint4(0, 0, 0, 0);
    int idx = threadIdx.x;
    for (int r = 0; r < reps; r++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint4 v = tile[(idx + k * PK_THREADS) & 2047];
            acc.x += v.x; acc.y ^= v.y; acc.z += v.z; acc.w ^= v.w;
        }
        idx = (idx + 32) & 2047;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) sink[0] = acc.x;
}

template <typename K>
float time_ms(cudaStream_t st, K launch, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a, st);
    for (int i = 0; i < reps; i++) launch();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / reps;
}

}  // namespace

extern "C" bdc_status bdc_measure_peaks(void *scratch_dev, size_t bytes, void *cuda_stream, double *out) {
    if (!scratch_dev || !out || bytes < ((size_t)64 << 20) || (((uintptr_t)scratch_dev) & 15)) {
        bdc_set_error("bdc_measure_peaks: need a 16-byte aligned device scratch buffer of at least 64 MiB");
        return BDC_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    BDC_CUDA_TRY(cudaGetDevice(&dev));
    BDC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 8;  // 8 CTAs of 256 threads per SM: 64 warps
    unsigned *sink = (unsigned *)scratch_dev;
    const double fma_ops = (double)grid * PK_THREADS * PK_CHAINS * PK_ITERS;
    float ms32 = time_ms(st, [&] { k_fma_rate<float><<<grid, PK_THREADS, 0, st>>>(1.0f, (float *)sink); }, 5);
    float ms64 = time_ms(st, [&] { k_fma_rate<double><<<grid, PK_THREADS, 0, st>>>(1.0, (double *)sink); }, 2);
    // L2: a 32 MiB buffer (far below the L2 size), read l2_reps times over by the grid
    const size_t l2_bytes = (size_t)32 << 20, words = l2_bytes / 16;
    const uint4 *buf = (const uint4 *)((char *)scratch_dev + 4096);
    BDC_CUDA_TRY(cudaMemsetAsync((void *)buf, 1, l2_bytes, st));
    const int l2_reps = 8;
    float msl2 = time_ms(st, [&] { k_l2_read<<<grid, PK_THREADS, 0, st>>>(buf, words, l2_reps, sink); }, 5);
    const int sm_reps = 4096;
    float mssm = time_ms(st, [&] { k_smem_rate<<<grid, PK_THREADS, 0, st>>>(sm_reps, sink); }, 5);
    BDC_CUDA_TRY(cudaGetLastError());
    BDC_CUDA_TRY(cudaStreamSynchronize(st));
    out[0] = fma_ops / (ms32 * 1e-3) / 1e12;  // FP32 FMA (or add) instructions per second, 1e12
    out[1] = fma_ops / (ms64 * 1e-3) / 1e12;  // FP64, same
    out[2] = (double)l2_bytes * l2_reps / (msl2 * 1e-3) / 1e9;  // L2 read GB/s
    out[3] = (double)grid * PK_THREADS * 8.0 * sm_reps * 16.0 / (mssm * 1e-3) / 1e12;  // shared memory TB/s
    out[4] = (double)sms;
    return BDC_OK;
}
