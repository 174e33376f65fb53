// Exact check of the tcgen05 main loop of the sliced products (tc_sliced.cuh): random signed
// digit planes (|d| <= 63, so every FP32 accumulator stays an exact integer), stored
// [S][rows][pitch] with pitch = K rounded up to 16 and zeros past K, addressed through one 2-D
// tensor map per operand; A rows past `arows` are zero.  Every accumulator of every digit order
// is compared with the integer sum_{k + l = g} A_k B_l^T computed on the host; the shapes are
// those of the chain (S = 6 and 5, N = 48) and pair (S = 5, N = 96) kernels, with one and with
// several K stages, two K chunks, and K not a multiple of 32.  Exit status 0 when every value
// matches.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include "../paper_2407_06409_gb300/csrc/tc_sliced.cuh"

bool tc_encode_map(CUtensorMap* map, const void* base, long long inner, long long pitch, long long rows, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess && q == cudaDriverEntryPointSuccess) encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  if (!encode) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, int NB>
__global__ void __launch_bounds__(256, 1) mainloop_check(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int K, double* out, int* status) {
  extern __shared__ unsigned char dyn[];
  __shared__ TcsBarriers bar;
  const uint32_t sbase = (tc_smem_u32(dyn) + 1023u) & ~1023u;
  const uint32_t tmem = tcs_setup(bar);
  const TcsTile A{&tA, 0, 128}, B{&tB, 0, NB};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane, cb = (warp >> 2) * (NB / 2);
  TcsProgress pr;
  const bool ok = tcs_mainloop<S, NB>(A, B, K, sbase, bar, 1LL << 32, pr, [&]() {
    for (int g = 0; g < S; ++g)
      for (int j8 = 0; j8 < NB / 16; ++j8) {
        float v[8];
        tc_ld8(tcs_lane_addr(tmem, g * NB + cb + j8 * 8), v);
        for (int i = 0; i < 8; ++i) out[((long long)g * 128 + row) * NB + cb + j8 * 8 + i] += (double)v[i];
      }
  });
  tcs_teardown(bar, !ok, pr, status);
}

static unsigned short bf(int v) {
  __nv_bfloat16 h = __float2bfloat16((float)v);
  return *reinterpret_cast<unsigned short*>(&h);
}

template <int S, int NB>
int run(int K, int arows) {
  std::vector<int> A((size_t)S * 128 * K), B((size_t)S * NB * K);
  for (auto& a : A) a = rand() % 127 - 63;
  for (auto& b : B) b = rand() % 127 - 63;
  const int P = (K + 15) / 16 * 16;
  for (int k = 0; k < S; ++k)
    for (int r = arows; r < 128; ++r)
      for (int j = 0; j < K; ++j) A[((size_t)k * 128 + r) * K + j] = 0;
  std::vector<unsigned short> Ah((size_t)S * 128 * P, 0), Bh((size_t)S * NB * P, 0);
  for (int k = 0; k < S; ++k)
    for (int r = 0; r < 128; ++r)
      for (int j = 0; j < K; ++j) Ah[((size_t)k * 128 + r) * P + j] = bf(A[((size_t)k * 128 + r) * K + j]);
  for (int k = 0; k < S; ++k)
    for (int r = 0; r < NB; ++r)
      for (int j = 0; j < K; ++j) Bh[((size_t)k * NB + r) * P + j] = bf(B[((size_t)k * NB + r) * K + j]);
  unsigned short *dA, *dB;
  double* dO;
  int* dS;
  cudaMalloc(&dA, Ah.size() * 2);
  cudaMalloc(&dB, Bh.size() * 2);
  cudaMalloc(&dO, sizeof(double) * S * 128 * NB);
  cudaMalloc(&dS, sizeof(int));
  cudaMemcpy(dA, Ah.data(), Ah.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, Bh.data(), Bh.size() * 2, cudaMemcpyHostToDevice);
  cudaMemset(dO, 0, sizeof(double) * S * 128 * NB);
  cudaMemset(dS, 0, sizeof(int));
  const int smem = TcsShape<S, NB>::kBytes;
  cudaFuncSetAttribute(mainloop_check<S, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CUtensorMap ta, tb;
  if (!tc_encode_map(&ta, dA, P, P, (long long)S * 128, 128) || !tc_encode_map(&tb, dB, P, P, (long long)S * NB, NB)) {
    printf("tensor map encode failed\n");
    return 3;
  }
  mainloop_check<S, NB><<<1, 256, smem>>>(ta, tb, K, dO, dS);
  cudaError_t e = cudaDeviceSynchronize();
  printf("S=%d NB=%d K=%d kernel: %s\n", S, NB, K, cudaGetErrorString(e));
  if (e != cudaSuccess) return 2;
  int st = 0;
  std::vector<double> O((size_t)S * 128 * NB);
  cudaMemcpy(&st, dS, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(O.data(), dO, sizeof(double) * O.size(), cudaMemcpyDeviceToHost);
  long bad = 0;
  int shown = 0;
  for (int g = 0; g < S; ++g)
    for (int r = 0; r < 128; ++r)
      for (int c = 0; c < NB; ++c) {
        double ref = 0;
        if (r < arows)
          for (int k = 0; k <= g; ++k)
            for (int j = 0; j < K; ++j) ref += (double)A[((size_t)k * 128 + r) * K + j] * B[((size_t)(g - k) * NB + c) * K + j];
        const double got = O[((size_t)g * 128 + r) * NB + c];
        if (got != ref) {
          ++bad;
          if (shown < 10) {
            printf("  mismatch g=%d r=%d c=%d got %.1f ref %.1f\n", g, r, c, got, ref);
            ++shown;
          }
        }
      }
  printf("  status %d mismatches %ld of %d\n", st, bad, S * 128 * NB);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dO);
  cudaFree(dS);
  return (bad == 0 && st == 0) ? 0 : 1;
}

int main() {
  srand(7);
  int rc = 0;
  rc |= run<6, 48>(288, 120);
  rc |= run<5, 48>(96, 128);
  rc |= run<5, 96>(144, 126);
  rc |= run<6, 48>(16, 7);
  rc |= run<6, 48>(448, 128);
  printf("%s\n", rc ? "FAILED" : "all exact");
  return rc;
}
