// Arithmetic-peak probes for the roofline denominators that MEASURED_PEAKS-style
// copy / BF16 GEMM measurements do not cover: FP64 FMA on the CUDA cores, FP64
// on the tensor path (mma.sync m8n8k4 f64), and FP32 FMA.  Each probe runs a loop
// of independent multiply-adds over every SM, timed with
// CUDA events on its own stream after a warm-up launch; the result is the best of
// `reps` timed launches in TFLOP/s (2 flop per multiply-add).
//
// Built as its own small library (not part of the eddy-current ABI).

#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int ACC = 16;  // independent accumulators per thread

__global__ void __launch_bounds__(256) dfma_loop(int iters, double seed, double* sink) {
  double a[ACC];
#pragma unroll
  for (int j = 0; j < ACC; ++j) a[j] = seed + threadIdx.x * 1e-9 + j;
  const double x = 0.999999, y = 1e-7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < ACC; ++j) a[j] = fma(a[j], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < ACC; ++j) s += a[j];
  if (s == 123.456) sink[blockIdx.x] = s;   // never true; keeps the loop alive
}

// FP64 FMAs fed from shared memory, the way a tiled product feeds them: each thread
// multiplies 4 shared values by 4 register values into 16 accumulators per step.
__global__ void __launch_bounds__(256) dfma_smem_loop(int iters, double seed, double* sink) {
  __shared__ double sh[4][256];
  for (int q = threadIdx.x; q < 4 * 256; q += 256) sh[q >> 8][q & 255] = seed + q * 1e-9;
  __syncthreads();
  double acc[16], b[4];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = 0.5 + (threadIdx.x + j) * 1e-9;
  for (int i = 0; i < iters; ++i) {
    double a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = sh[q][(threadIdx.x + i) & 255];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[q * 4 + j] = fma(a[q], b[j], acc[q * 4 + j]);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += acc[j];
  if (s == 123.456) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma_loop(int iters, float seed, float* sink) {
  float a[ACC];
#pragma unroll
  for (int j = 0; j < ACC; ++j) a[j] = seed + threadIdx.x * 1e-6f + j;
  const float x = 0.9999f, y = 1e-4f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < ACC; ++j) a[j] = fmaf(a[j], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < ACC; ++j) s += a[j];
  if (s == 123.456f) sink[blockIdx.x] = s;
}

// One warp-wide D = A B + C per instruction, m8n8k4 with FP64 operands: each lane
// holds one A element, one B element and two accumulator elements.  Four
// independent accumulator pairs per lane.
__global__ void __launch_bounds__(256) dmma_loop(int iters, double seed, double* sink) {
  const double av = seed + (threadIdx.x & 31) * 1e-9, bv = 0.5 + (threadIdx.x & 7) * 1e-9;
  double c[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    c[j][0] = 0.0;
    c[j][1] = 0.0;
  }
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
          : "+d"(c[j][0]), "+d"(c[j][1])
          : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  if (s == 123.456) sink[blockIdx.x] = s;
}

// Both FP64 paths at once: even warps run the FMA loop, odd warps the mma.sync loop.
// If the two share one unit the combined rate equals either alone; if they are separate
// it approaches their sum.
__global__ void __launch_bounds__(256) mixed64_loop(int iters, double seed, double* sink) {
  const int w = threadIdx.x >> 5;
  double s = 0.0;
  if ((w & 1) == 0) {
    double a[ACC];
#pragma unroll
    for (int j = 0; j < ACC; ++j) a[j] = seed + threadIdx.x * 1e-9 + j;
    const double x = 0.999999, y = 1e-7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < ACC; ++j) a[j] = fma(a[j], x, y);
    }
#pragma unroll
    for (int j = 0; j < ACC; ++j) s += a[j];
  } else {
    const double av = seed + (threadIdx.x & 31) * 1e-9, bv = 0.5 + (threadIdx.x & 7) * 1e-9;
    double c[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      c[j][0] = 0.0;
      c[j][1] = 0.0;
    }
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
            : "+d"(c[j][0]), "+d"(c[j][1])
            : "d"(av), "d"(bv));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  }
  if (s == 123.456) sink[blockIdx.x] = s;
}

template <typename F>
double best_ms(F launch, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();   // warm-up
  cudaDeviceSynchronize();
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace

// out[0] FP64 FMA TFLOP/s (the faster of a register-operand loop and a shared-memory
// fed loop), out[1] FP64 mma.sync TFLOP/s, out[2] FP32 FMA TFLOP/s,
// out[3] SM count, out[4] SM clock the device reports (MHz), out[5] FP64 TFLOP/s with
// half the warps on each FP64 path at once.  Returns 0 on success, else the CUDA error
// code.
extern "C" int ec_peak_probe(int reps, double* out) {
  if (!out || reps < 1) return 1;
  int dev = 0, sms = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 65536) != cudaSuccess) return (int)cudaGetLastError();
  const int blocks = sms * 8, threads = 256;
  const int it64 = 2048, it32 = 32768, itmma = 2048;
  const double fl64 = 2.0 * ACC * (double)it64 * blocks * threads;
  const double fl32 = 2.0 * ACC * (double)it32 * blocks * threads;
  const double flmma = 2.0 * 8 * 8 * 4 * 4.0 * (double)itmma * blocks * (threads / 32);
  const double t64r = best_ms([&] { dfma_loop<<<blocks, threads>>>(it64, 1.0, sink); }, reps);
  const double t64s = best_ms([&] { dfma_smem_loop<<<blocks, threads>>>(it64, 1.0, sink); }, reps);
  // both variants do 2 * 16 * it64 flop per thread: the faster one sets the peak
  const double t64 = t64r < t64s ? t64r : t64s;
  const double tmma = best_ms([&] { dmma_loop<<<blocks, threads>>>(itmma, 1.0, sink); }, reps);
  const double t32 = best_ms(
      [&] { ffma_loop<<<blocks, threads>>>(it32, 1.0f, reinterpret_cast<float*>(sink)); }, reps);
  // mixed: half the warps do fl64 / 2 of FMA work, half do flmma / 2 of mma work
  const double tmix =
      best_ms([&] { mixed64_loop<<<blocks, threads>>>(it64, 1.0, sink); }, reps);
  const double flmix = 0.5 * fl64 + 0.5 * (2.0 * 8 * 8 * 4 * 4.0 * (double)it64 * blocks * (threads / 32));
  const cudaError_t e = cudaGetLastError();
  cudaFree(sink);
  if (e != cudaSuccess) return (int)e;
  out[0] = fl64 / (t64 * 1e-3) / 1e12;
  out[1] = flmma / (tmma * 1e-3) / 1e12;
  out[2] = fl32 / (t32 * 1e-3) / 1e12;
  out[3] = sms;
  out[4] = clk / 1000.0;
  out[5] = flmix / (tmix * 1e-3) / 1e12;
  return 0;
}
