// Tensor-core (tcgen05) BF16 GEMM tile with the FP32 accumulator in TMEM.
//
// C[M x N] = A[M x K] B[K x N]: A row-major BF16 (K contiguous), B given as
// its transpose Bt[N x K] (K contiguous), C row-major FP32.  Each CTA of 128
// threads computes 128 rows: it stages its A rows and all of Bt in shared
// memory in the no-swizzle K-major core-matrix layout, one thread issues
// K/16 tcgen05.mma instructions (M = 128, N, K = 16) into a TMEM
// accumulator, tcgen05.commit arrives on an mbarrier, and each warp reads
// its 32 accumulator lanes back with tcgen05.ld.  This is the building block
// of the implicit-GEMM convolutions; tpfa_tc_gemm_bf16 exposes it so that
// its numerics can be checked on its own.
#include "tc_common.cuh"
#include "tpfa_internal.cuh"

namespace tpfa {
namespace {

constexpr uint32_t kWaitLimit = 1u << 20;  // mbarrier polls before giving up

template <int N>
__global__ void __launch_bounds__(128)
tc_gemm_kernel(const uint16_t* __restrict__ A, const uint16_t* __restrict__ Bt,
               float* __restrict__ C, int M, int K, int* err) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  constexpr uint32_t kCols = N < 32 ? 32 : N;  // TMEM columns: power of two >= 32
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  unsigned char* sA = sm;
  unsigned char* sB = sm + (size_t)128 * K * 2;
  const int kc = K / 8;  // 16-byte chunks per row
  for (int idx = threadIdx.x; idx < 128 * kc; idx += 128) {
    const int r = idx / kc, c = idx % kc;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (m0 + r < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + c * 8);
    *reinterpret_cast<uint4*>(sA + tc::kmajor_off(r, c * 8, K)) = v;
  }
  for (int idx = threadIdx.x; idx < N * kc; idx += 128) {
    const int r = idx / kc, c = idx % kc;
    *reinterpret_cast<uint4*>(sB + tc::kmajor_off(r, c * 8, K)) =
        *reinterpret_cast<const uint4*>(Bt + (size_t)r * K + c * 8);
  }
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  if (warp == 0) tc::tmem_alloc(&tbase, kCols);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t d = tbase;
  if (threadIdx.x == 0) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N);
    for (int s = 0; s < K / 16; ++s) {
      const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + s * 256, 128, sbo);
      const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + s * 256, 128, sbo);
      tc::mma_bf16(d, ad, bd, idesc, s > 0);
    }
    tc::mma_commit(&bar);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar, 0, kWaitLimit));
  tc::fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8];
      tc::tmem_ld8(d + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (row < M) {
#pragma unroll
        for (int i = 0; i < 8; ++i) C[(size_t)row * N + c0 + i] = v[i];
      }
    }
  } else if (lane == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(d, kCols);
}

template <int N>
cudaError_t launch_gemm(const uint16_t* A, const uint16_t* Bt, float* C, int M, int K, int* err,
                        cudaStream_t s) {
  const int smem = (128 + N) * K * 2;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<N><<<(M + 127) / 128, 128, smem, s>>>(A, Bt, C, M, K, err);
  return cudaGetLastError();
}

}  // namespace
}  // namespace tpfa

extern "C" int tpfa_tc_gemm_bf16(const uint16_t* A, const uint16_t* Bt, float* C, int M, int N,
                                 int K, void* stream) {
  using namespace tpfa;
  if (M < 1 || K < 16 || K > 256 || K % 16 != 0) return TPFA_EINVAL;
  if (N != 16 && N != 32 && N != 64 && N != 128) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  if (!dev_ok(A, (size_t)M * K * 2, 16, dev) || !dev_ok(Bt, (size_t)N * K * 2, 16, dev) ||
      !dev_ok(C, (size_t)M * N * 4, 16, dev))
    return TPFA_EINVAL;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return TPFA_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = TPFA_OK;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    switch (N) {
      case 16: e = launch_gemm<16>(A, Bt, C, M, K, err, s); break;
      case 32: e = launch_gemm<32>(A, Bt, C, M, K, err, s); break;
      case 64: e = launch_gemm<64>(A, Bt, C, M, K, err, s); break;
      default: e = launch_gemm<128>(A, Bt, C, M, K, err, s); break;
    }
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = TPFA_ECUDA;
  } else if (herr) {
    rc = TPFA_EINTERNAL;
  }
  cudaFree(err);
  return rc;
}
