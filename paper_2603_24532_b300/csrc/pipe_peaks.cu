// Pipe throughput probes on one GPU: FP64/FP32/MUFU/INT/conversion/shared atomics, register-only
// work and one store per thread.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_peaks paper_2603_24532_b300/csrc/pipe_peaks.cu && ./pipe_peaks
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int OP>
__global__ void k_op(double* out, int iters, double seed) {
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[8]; float f[8]; unsigned u[8];
  for (int j = 0; j < 8; ++j) { a[j] = seed + gid * 1e-9 + j * 1e-3; f[j] = (float)a[j]; u[j] = gid * 2654435761u + j; }
  double b = 1.0000001, c = 1e-7;
  float fb = 1.0000001f, fc = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (OP == 0) a[j] = fma(a[j], b, c);              // DFMA
      if (OP == 1) a[j] = a[j] + c;                     // DADD
      if (OP == 2) f[j] = fmaf(f[j], fb, fc);           // FFMA
      if (OP == 3) f[j] = exp2f(f[j]) * 0.5f;           // MUFU.EX2 (+FMUL)
      if (OP == 4) a[j] = sqrt(a[j]) + c;               // FP64 sqrt
      if (OP == 5) a[j] = 1.0 / a[j] + c;               // FP64 reciprocal/div
      if (OP == 6) { u[j] = __umulhi(u[j], 0xD2511F53u) ^ u[j]; }  // IMAD.HI + LOP
      if (OP == 7) a[j] = a[j] + (double)(u[j] + it);   // I2F.F64 + DADD
      if (OP == 8) f[j] = f[j] + (float)a[j];           // F2F.F32.F64 + FADD
      if (OP == 9) { double s, co; sincospi(a[j], &s, &co); a[j] = s + co * c; }  // FP64 sincospi
      if (OP == 10) a[j] = exp(-a[j]) + c;              // FP64 exp
      if (OP == 11) { f[j] = __frcp_rn(f[j]) + fc; }    // FP32 rcp
    }
  }
  double s = 0; for (int j = 0; j < 8; ++j) s += a[j] + f[j] + (double)u[j];
  out[gid] = s;
}

template<int OP>
__global__ void k_atom(double* out, int iters) {
  __shared__ double hd[1024];
  __shared__ float hf[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) { hd[i] = 0; hf[i] = 0; }
  __syncthreads();
  unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    x = x * 1664525u + 1013904223u;
    unsigned idx = x >> 22;  // 0..1023
    if (OP == 0) atomicAdd(&hd[idx], 1.0);
    if (OP == 1) atomicAdd(&hf[idx], 1.0f);
    if (OP == 2) atomicAdd((unsigned long long*)&hd[idx], 1ull);
  }
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = hd[0] + hf[0];
}

template<class K>
float timeit(K kern, int blocks, int threads, double* out, int iters) {
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  kern<<<blocks, threads>>>(out, iters, 1.0);
  cudaEventRecord(a);
  kern<<<blocks, threads>>>(out, iters, 1.0);
  cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms, a, b); return ms;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("%s SMs=%d clockKHz=%d smem/block optin=%zu regs/SM=%d\n", p.name, p.multiProcessorCount, clk, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  int sms = p.multiProcessorCount;
  double* out; CK(cudaMalloc(&out, sizeof(double) * sms * 8 * 1024));
  const char* names[] = {"DFMA", "DADD", "FFMA", "EX2f", "DSQRT", "DRCP(1/x)", "IMULHI+XOR", "I2F64+DADD", "F2F32+FADD", "DSINCOSPI", "DEXP", "FRCP"};
  int iters[] = {2000, 2000, 200000, 20000, 200, 200, 50000, 2000, 20000, 100, 100, 20000};
  for (int op = 0; op < 12; ++op) {
    for (int tpb : {256, 512}) {
      int blocks = sms * (1024 / tpb) * 2;
      float ms = 0;
      switch (op) {
        case 0: ms = timeit(k_op<0>, blocks, tpb, out, iters[op]); break;
        case 1: ms = timeit(k_op<1>, blocks, tpb, out, iters[op]); break;
        case 2: ms = timeit(k_op<2>, blocks, tpb, out, iters[op]); break;
        case 3: ms = timeit(k_op<3>, blocks, tpb, out, iters[op]); break;
        case 4: ms = timeit(k_op<4>, blocks, tpb, out, iters[op]); break;
        case 5: ms = timeit(k_op<5>, blocks, tpb, out, iters[op]); break;
        case 6: ms = timeit(k_op<6>, blocks, tpb, out, iters[op]); break;
        case 7: ms = timeit(k_op<7>, blocks, tpb, out, iters[op]); break;
        case 8: ms = timeit(k_op<8>, blocks, tpb, out, iters[op]); break;
        case 9: ms = timeit(k_op<9>, blocks, tpb, out, iters[op]); break;
        case 10: ms = timeit(k_op<10>, blocks, tpb, out, iters[op]); break;
        case 11: ms = timeit(k_op<11>, blocks, tpb, out, iters[op]); break;
      }
      CK(cudaGetLastError());
      double ops = (double)blocks * tpb * iters[op] * 8;
      printf("%-12s tpb=%d  %.3f ms  %.4g op/s  %.3f op/clk/SM@maxclk\n", names[op], tpb, ms, ops / (ms * 1e-3),
             ops / (ms * 1e-3) / (sms * clk * 1e3));
    }
  }
  const char* an[] = {"ATOMS.F64", "ATOMS.F32", "ATOMS.U64"};
  for (int op = 0; op < 3; ++op) {
    int blocks = sms * 4, tpb = 256, it = 20000;
    cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(a);
      if (op == 0) k_atom<0><<<blocks, tpb>>>(out, it);
      if (op == 1) k_atom<1><<<blocks, tpb>>>(out, it);
      if (op == 2) k_atom<2><<<blocks, tpb>>>(out, it);
      cudaEventRecord(b); cudaEventSynchronize(b);
    }
    CK(cudaGetLastError());
    float ms; cudaEventElapsedTime(&ms, a, b);
    double ops = (double)blocks * tpb * it;
    printf("%-12s %.3f ms  %.4g op/s  %.3f op/clk/SM\n", an[op], ms, ops / (ms * 1e-3), ops / (ms * 1e-3) / (sms * clk * 1e3));
  }
  CK(cudaDeviceSynchronize());
  return 0;
}
