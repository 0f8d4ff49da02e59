// Launch/dispatch of the stage kernel for one storage precision (included by stage_f*.cu so
// that the precisions compile in parallel).
#pragma once

#include <algorithm>
#include <cstdlib>
#include <map>

#include "dwf_internal.h"

namespace dwf {

template <int P, int LS, bool DAG, bool BLK, int POST, int MINB>
static cudaError_t stage_launch_v(const StageArgs& b, size_t sm, long g, cudaStream_t st) {
  auto k = stage_kernel<P, LS, DAG, BLK, POST, MINB>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k<<<dim3((unsigned)g), dim3(32, LS), sm, st>>>(b);
  return cudaGetLastError();
}

// Online autotuner of the register budget (2 or 3 resident CTAs per SM): the first launches
// of each (kernel, problem size) alternate between the two variants bracketed by CUDA
// events; once both have been timed twice the faster one is used for good.  The timed
// launches are the caller's real work, so tuning costs nothing extra.  Tuning happens
// outside stream capture only (a captured launch uses the current choice).
struct StageTune {
  int next = 0;          // launches recorded so far
  int chosen = -1;       // decided variant (0: 2 CTAs/SM, 1: 3 CTAs/SM)
  cudaEvent_t ev[8] = {};
  bool pending = false;
};

template <int P, int LS, bool DAG, bool BLK, int POST>
static cudaError_t stage_launch_post(const StageArgs& a, cudaStream_t st) {
  const size_t sm = stage_smem_bytes<P>(LS, POST);
  StageArgs b = a;
  if (b.ntiles == 0) b.ntiles = b.Vp / 32;
  const long g = b.grid > 0 ? std::min<long>(b.grid, b.ntiles) : b.ntiles;
  static std::map<long, StageTune> tunes;   // per tile count
  StageTune& T = tunes[b.ntiles];
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  const bool capturing = (cap != cudaStreamCaptureStatusNone);
  // event queries are not allowed while the stream is being captured: decide only outside
  if (!capturing && T.chosen < 0 && T.next >= 4 && T.pending) {
    // decide once every timed launch has completed
    bool done = true;
    for (int i = 0; i < 8; i++) done = done && cudaEventQuery(T.ev[i]) == cudaSuccess;
    cudaGetLastError();
    if (done) {
      float t[4];
      for (int i = 0; i < 4; i++) cudaEventElapsedTime(&t[i], T.ev[2 * i], T.ev[2 * i + 1]);
      T.chosen = (t[1] + t[3] < t[0] + t[2]) ? 1 : 0;
      for (auto& e : T.ev) cudaEventDestroy(e);
      T.pending = false;
    }
  }
  const char* force = getenv("DWF_STAGE_VARIANT");
  int v = T.chosen >= 0 ? T.chosen : 0;
  if (force && (force[0] == '0' || force[0] == '1')) {
    v = force[0] - '0';
  } else if (T.chosen < 0 && T.next < 4 && !capturing) {
    if (T.next == 0)
      for (auto& e : T.ev) cudaEventCreate(&e);
    v = T.next & 1;
    cudaEventRecord(T.ev[2 * T.next], st);
    cudaError_t e = v ? stage_launch_v<P, LS, DAG, BLK, POST, 3>(b, sm, g, st)
                      : stage_launch_v<P, LS, DAG, BLK, POST, 2>(b, sm, g, st);
    cudaEventRecord(T.ev[2 * T.next + 1], st);
    T.next++;
    T.pending = true;
    return e;
  }
  return v ? stage_launch_v<P, LS, DAG, BLK, POST, 3>(b, sm, g, st)
           : stage_launch_v<P, LS, DAG, BLK, POST, 2>(b, sm, g, st);
}

template <int P, int LS, bool DAG, bool BLK>
static cudaError_t stage_launch_one(const StageArgs& a, cudaStream_t st) {
  if (!a.post) return stage_launch_post<P, LS, DAG, BLK, 0>(a, st);
  if (a.post_sparse) return stage_launch_post<P, LS, DAG, BLK, 3>(a, st);
  if constexpr (P == P64 || P == P32) {
    if (a.post_struct) return stage_launch_post<P, LS, DAG, BLK, 4>(a, st);
  }
  if constexpr (P == P16 || P == PB16) {
    if (a.post_h) return stage_launch_post<P, LS, DAG, BLK, 2>(a, st);
  }
  return stage_launch_post<P, LS, DAG, BLK, 1>(a, st);
}

template <int P, int LS>
static cudaError_t stage_dispatch_ls(const StageArgs& a, bool dag, bool blocked,
                                     cudaStream_t st) {
  if (dag)
    return blocked ? stage_launch_one<P, LS, true, true>(a, st)
                   : stage_launch_one<P, LS, true, false>(a, st);
  return blocked ? stage_launch_one<P, LS, false, true>(a, st)
                 : stage_launch_one<P, LS, false, false>(a, st);
}

template <int P>
cudaError_t launch_stage(const StageArgs& a, int Ls, bool dag, bool blocked, cudaStream_t st) {
  switch (Ls) {
    case 4: return stage_dispatch_ls<P, 4>(a, dag, blocked, st);
    case 6: return stage_dispatch_ls<P, 6>(a, dag, blocked, st);
    case 8: return stage_dispatch_ls<P, 8>(a, dag, blocked, st);
    case 10: return stage_dispatch_ls<P, 10>(a, dag, blocked, st);
    case 12: return stage_dispatch_ls<P, 12>(a, dag, blocked, st);
    case 16: return stage_dispatch_ls<P, 16>(a, dag, blocked, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dwf
