// Batched solver: a chunk of FP32 CG steps of every problem of one Ls group in a single
// persistent, cooperative launch.  Each step is five phases over all tiles of all problems
// (stage A, stage B with the per-problem <p, A p> -> alpha, stage A^dag, stage B^dag with
// r -= alpha q and ||r||^2 -> beta and the convergence flags, then x += alpha p, p = r + beta
// p, u = D+ p), separated by grid barriers with bounded waits.  The per-problem reductions
// are the stage kernels' segmented ones (the last tile of a problem finalises its scalars);
// tiles of converged problems skip every phase.  Data written in the launch is read through
// L2 (coherent loads); links, tables and per-problem parameters through the read-only path.
#include "dwf_internal.h"
#include "sync.cuh"
#include "vec_tile.cuh"

namespace dwf {

template <int LS, int G>
__global__ void __launch_bounds__(32 * LS, LS >= 16 ? 1 : 2) batch_cg_kernel(const BatchStepArgs b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red_scratch[32];
  __shared__ uint64_t tc_mbar;
  __shared__ uint32_t tc_slot;
  __shared__ uint64_t lk_mbar;
  if constexpr (gather_tma(G)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) tc::mbar_init(&lk_mbar, 1);
    __syncthreads();
  }
  uint32_t tc_phase = 0, lk_phase = 0;
  unsigned nbar = 0;
  const unsigned C = gridDim.x;
  auto barrier = [&]() -> bool {
    ++nbar;
    return slot_barrier(b.bar, nbar * C, b.wait_ns, b.err);
  };
  for (int k = 0; k < b.nsteps; k++) {
    for (long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      if (!stage_tile<P32, LS, false, false, 4, G, SP_ONE, true>(
              b.A, t, smem_raw, red_scratch, &tc_mbar, &tc_slot, tc_phase, &lk_mbar, lk_phase))
        return;
      __syncthreads();
    }
    if (!barrier()) return;
    for (long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      if (!stage_tile<P32, LS, false, false, 0, G, SP_ONE, true>(
              b.B, t, smem_raw, red_scratch, &tc_mbar, &tc_slot, tc_phase, &lk_mbar, lk_phase))
        return;
      __syncthreads();
    }
    if (!barrier()) return;
    for (long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      if (!stage_tile<P32, LS, true, false, 4, G, SP_ONE, true>(
              b.Ad, t, smem_raw, red_scratch, &tc_mbar, &tc_slot, tc_phase, &lk_mbar, lk_phase))
        return;
      __syncthreads();
    }
    if (!barrier()) return;
    for (long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      if (!stage_tile<P32, LS, true, false, 3, G, SP_ONE, true>(
              b.Bd, t, smem_raw, red_scratch, &tc_mbar, &tc_slot, tc_phase, &lk_mbar, lk_phase))
        return;
      __syncthreads();
    }
    if (!barrier()) return;
    for (long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      vec_tile<P32, LS, true>(b.U, t, (unsigned)b.ntiles, smem_raw);
      __syncthreads();
    }
    if (!barrier()) return;
  }
}

template <int LS, int G>
static size_t batch_smem() {
  size_t m = (size_t)LS * 24 * 32 * sizeof(float);   // the update's slice exchange
  const int posts[3] = {4, 0, 3};
  for (int post : posts) m = std::max(m, stage_smem_bytes<P32>(LS, post, G));
  return m;
}

template <int LS, int G>
static cudaError_t batch_launch_lg(const BatchStepArgs& b, int grid, int* cap, int nsm,
                                   cudaStream_t st, bool query) {
  auto k = batch_cg_kernel<LS, G>;
  const size_t smem = batch_smem<LS, G>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (query) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * LS, smem);
    if (e != cudaSuccess) return e;
    *cap = per_sm * nsm;
    return cudaSuccess;
  }
  // a cooperative launch through the extensible API (capturable in a CUDA graph)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(32, LS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, b);
}

template <int LS>
static cudaError_t batch_launch_l(const BatchStepArgs& b, int gather, int grid, int* cap,
                                  int nsm, cudaStream_t st, bool query) {
  return gather == G_TMA ? batch_launch_lg<LS, G_TMA>(b, grid, cap, nsm, st, query)
                         : batch_launch_lg<LS, G_REG>(b, grid, cap, nsm, st, query);
}

cudaError_t batch_steps_launch(const BatchStepArgs& b, int Ls, int gather, int grid, int* cap,
                               int nsm, cudaStream_t st, bool query) {
  switch (Ls) {
    case 4: return batch_launch_l<4>(b, gather, grid, cap, nsm, st, query);
    case 6: return batch_launch_l<6>(b, gather, grid, cap, nsm, st, query);
    case 8: return batch_launch_l<8>(b, gather, grid, cap, nsm, st, query);
    case 10: return batch_launch_l<10>(b, gather, grid, cap, nsm, st, query);
    case 12: return batch_launch_l<12>(b, gather, grid, cap, nsm, st, query);
    case 16: return batch_launch_l<16>(b, gather, grid, cap, nsm, st, query);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dwf
