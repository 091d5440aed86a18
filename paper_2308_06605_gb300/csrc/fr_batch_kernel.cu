// One variant of the batched persistent stage kernel (the stage of every case of an ensemble in
// one cooperative launch; phases separated by bounded grid barriers, see fr_bodies.cuh).  This
// file is compiled once per variant with FRX_BATCH_MIXED (0: FP64, 1: double-float) and
// FRX_BATCH_BLOCK (256 or 512 threads) defined, so the four variants build in parallel; each
// variant exports its launch, occupancy and basis-upload functions under suffixed names.
#include "fr_bodies.cuh"

#if !defined(FRX_BATCH_MIXED) || !defined(FRX_BATCH_BLOCK)
#error "compile with -DFRX_BATCH_MIXED=0|1 -DFRX_BATCH_BLOCK=256|512"
#endif

#define FRX_BV_NAME2(base, m, b) base##_m##m##_b##b
#define FRX_BV_NAME(base, m, b) FRX_BV_NAME2(base, m, b)
#define FRX_BV(base) FRX_BV_NAME(base, FRX_BATCH_MIXED, FRX_BATCH_BLOCK)

namespace frx {

namespace {
using BatchT = std::conditional<FRX_BATCH_MIXED != 0, df32, double>::type;
constexpr int kBlock = FRX_BATCH_BLOCK;
}  // namespace

cudaError_t FRX_BV(batch_launch)(const BatchLaunch &L, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(k_batch_stage<BatchT, kBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BatchLaunch arg = L;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)k_batch_stage<BatchT, kBlock>, dim3(grid), dim3(kBlock), args, smem,
                                     st);
}

cudaError_t FRX_BV(batch_occupancy)(size_t smem, int *nb) {
  cudaError_t e =
      cudaFuncSetAttribute(k_batch_stage<BatchT, kBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_batch_stage<BatchT, kBlock>, kBlock, smem);
}

cudaError_t FRX_BV(batch_upload)() { return upload_basis_local(); }

}  // namespace frx
