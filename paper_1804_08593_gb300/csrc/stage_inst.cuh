// Launch of the stage kernel variants and their online autotuner (included by stage_ls.cu,
// which is compiled once per storage precision and Ls).
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "dwf_internal.h"

namespace dwf {

// the current device's ordinal (host state below is kept per device)
static int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

template <int P, int LS, bool DAG, bool BLK, int POST, int MINB, int G, int SP = 1>
static cudaError_t stage_launch_v(const StageArgs& b, size_t sm, long g, cudaStream_t st) {
  auto k = stage_kernel<P, LS, DAG, BLK, POST, MINB, G, SP>;
  static std::atomic<uint64_t> attr_set{0};   // one bit per device
  const int dev = current_device();
  const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
  if (!(attr_set.load() & bit)) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit);
  }
  k<<<dim3((unsigned)g), dim3(32, LS / slices_per_thread(SP)), sm, st>>>(b);
  return cudaGetLastError();
}

// Online autotuner over the launch variants of one stage (register budget for 2 or 3
// resident CTAs per SM and, where both apply, tensor-core or recurrence post): the first
// launches of each (stage kind, problem size) cycle through the candidates bracketed by CUDA
// events; once every candidate has been timed twice the fastest is used for good.  The timed
// launches are the caller's real work, so tuning costs nothing extra.  Tuning happens outside
// stream capture only (a captured launch uses the current choice), and only on launches
// without a stop flag; until a kind is decided, other launches use the first candidate.
using StageFn = cudaError_t (*)(const StageArgs&, size_t, long, cudaStream_t);
struct StageCand {
  StageFn fn;
  size_t smem;
  int per_sm;            // 0: one CTA per tile; k: persistent grid of k CTAs per SM
  int post, minb, gather, sp;  // for the tuning log
};
constexpr int MAX_CANDS = 12;
constexpr int TUNE_ROUNDS = 2;   // timed rounds after one untimed round (first-launch costs)
struct StageTune {
  int next = 0;          // launches recorded so far
  int chosen = -1;       // decided candidate
  cudaEvent_t ev[2 * TUNE_ROUNDS * MAX_CANDS] = {};
  bool pending = false;
};

// The variants timed per stage kind (the first is the default for launches that are never
// timed).  FP32 gathers into registers, plain or after a bulk L2 prefetch of the tile's links
// (and streamed inputs), or with the tile's links copied into shared memory by the TMA engine,
// with one or two fifth-dimension slices per thread; a register budget for 3 CTAs per SM
// spills, and the cp.async ring, per-direction L1 prefetch, prefetching the neighbour runs and
// prefetching the next tile of a persistent CTA measured slower.  FP16/BF16 gather through the
// L1-cached cp.async ring with a register budget for 2 or 3 CTAs per SM, with the tile's links
// and streams prefetched into L2 or its links staged in shared memory by TMA, one CTA per tile
// (persistent grids measured 10-35 % slower there; only the tensor-core post, whose set-up is
// per CTA, has them).  FP32 and FP64 (ALU bound): one CTA per tile or a persistent grid.
template <int P, int LS, bool DAG, bool BLK, int POST, int MINB, int G, int SP = 1>
static void stage_cand(StageCand* c, int& n, int per_sm) {
  c[n++] = {stage_launch_v<P, LS, DAG, BLK, POST, MINB, G, SP>,
            stage_smem_bytes<P>(LS, POST, G), per_sm, POST, MINB, G, SP};
}
template <int P, int LS, bool DAG, bool BLK, int POST>
static void stage_cands(StageCand* c, int& n) {
  constexpr bool H16 = (P == P16 || P == PB16);
  if constexpr (POST == 1) {
    // dense CUDA-core post: only where the recurrence is unstable or switched off
    stage_cand<P, LS, DAG, BLK, POST, 2, H16 ? G_RING : G_REG>(c, n, 0);
  } else if constexpr (POST == 2) {
    // tensor-core post: TMEM and the B operands are set up once per CTA, so a persistent
    // grid pays off
    stage_cand<P, LS, DAG, BLK, POST, 2, G_RING>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 3, G_RING>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_RING>(c, n, 2);
    stage_cand<P, LS, DAG, BLK, POST, 3, G_RING>(c, n, 3);
  } else if constexpr (H16) {
    // up to Ls = 12 a budget for 3 CTAs per SM (56 registers) wins; beyond, it spills
    constexpr int MB = LS <= 12 ? 3 : 2;
    stage_cand<P, LS, DAG, BLK, POST, MB, G_RING>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 5 - MB, G_RING>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, MB, G_RING_BPF>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, MB, G_RING_TMA>(c, n, 0);
  } else if constexpr (P == P32) {
    stage_cand<P, LS, DAG, BLK, POST, 2, G_BPF_L>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_REG>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_BPF_LS>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA>(c, n, 2);
    // two slices per thread, one link load for both (half the warps, twice the loads each)
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA, SP_PAIR>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA, SP_PAIR>(c, n, 2);
    // the same with the pairs packed in float2 (f32x2 arithmetic)
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA, SP_PAIR_F2>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_TMA, SP_PAIR_F2>(c, n, 2);
  } else {
    stage_cand<P, LS, DAG, BLK, POST, 2, G_REG>(c, n, 0);
    stage_cand<P, LS, DAG, BLK, POST, 2, G_REG>(c, n, 2);
  }
}

static int sm_count() {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, current_device()) !=
          cudaSuccess || n <= 0)
    n = 1;
  return n;
}

template <int P, int LS, bool DAG, bool BLK>
static cudaError_t stage_launch_one(const StageArgs& a, cudaStream_t st) {
  constexpr bool H16 = (P == P16 || P == PB16);
  StageCand c[MAX_CANDS];
  int n = 0, kind;
  if (!a.post) {
    kind = 0;
    stage_cands<P, LS, DAG, BLK, 0>(c, n);
  } else if (a.post_sparse) {
    kind = 3;
    stage_cands<P, LS, DAG, BLK, 3>(c, n);
  } else if (H16 && a.post_h && a.post_struct == 2) {
    kind = 5;
    if constexpr (H16) {
      stage_cands<P, LS, DAG, BLK, 2>(c, n);
      stage_cands<P, LS, DAG, BLK, 4>(c, n);
    }
  } else if (a.post_struct) {
    kind = 4;
    stage_cands<P, LS, DAG, BLK, 4>(c, n);
  } else if (H16 && a.post_h) {
    kind = 2;
    if constexpr (H16) stage_cands<P, LS, DAG, BLK, 2>(c, n);
  } else {
    kind = 1;
    stage_cands<P, LS, DAG, BLK, 1>(c, n);
  }
  StageArgs b = a;
  if (b.ntiles == 0) b.ntiles = b.Vp / 32;
  // an explicit grid (batched solver) is kept; otherwise the candidate decides
  auto grid_of = [&](const StageCand& k) -> long {
    if (b.grid > 0) return std::min<long>(b.grid, b.ntiles);
    return k.per_sm ? std::min<long>((long)k.per_sm * sm_count(), b.ntiles) : b.ntiles;
  };
  // failure-detection probe: a variant with TMA link staging, outside the tuner (FP64 stages
  // have none and refuse)
  if (b.wait_probe) {
    for (int k = 0; k < n; k++)
      if (gather_tma(c[k].gather)) return c[k].fn(b, c[k].smem, grid_of(c[k]), st);
    return cudaErrorNotSupported;
  }
  // per (device, tile count, kind); handles on different host threads share it
  static std::mutex mu;
  static std::map<std::tuple<int, long, int>, StageTune> tunes;
  std::lock_guard<std::mutex> lock(mu);
  StageTune& T = tunes[std::make_tuple(current_device(), b.ntiles, kind)];
  const int nt = TUNE_ROUNDS * n;                           // timed launches
  const int nl = nt + n;                                    // tuning launches
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  const bool capturing = (cap != cudaStreamCaptureStatusNone);
  // event queries are not allowed while the stream is being captured: decide only outside
  if (!capturing && T.chosen < 0 && T.next >= nl && T.pending) {
    bool done = true;
    for (int i = 0; i < 2 * nt; i++) done = done && cudaEventQuery(T.ev[i]) == cudaSuccess;
    cudaGetLastError();
    if (done) {
      float best = 0.f, tks[MAX_CANDS];
      for (int k = 0; k < n; k++) {
        float tk = 0.f;
        for (int i = k; i < nt; i += n) {
          float t = 0.f;
          cudaEventElapsedTime(&t, T.ev[2 * i], T.ev[2 * i + 1]);
          tk += t;
        }
        tks[k] = tk;
        if (T.chosen < 0 || tk < best) {
          best = tk;
          T.chosen = k;
        }
      }
      if (getenv("DWF_TUNE_LOG")) {   // one line per decision: every candidate's time
        fprintf(stderr, "dwf tune P%d Ls%d dag%d blk%d tiles %ld:", P, LS, (int)DAG, (int)BLK,
                b.ntiles);
        for (int k = 0; k < n; k++)
          fprintf(stderr, " %s[post%d minb%d gather%d sp%d sm%d %.1fus]", k == T.chosen ? "*" : "",
                  c[k].post, c[k].minb, c[k].gather, c[k].sp, c[k].per_sm,
                  1000.f * tks[k] / TUNE_ROUNDS);
        fprintf(stderr, "\n");
      }
      for (auto& e : T.ev)
        if (e) cudaEventDestroy(e);
      T.pending = false;
    }
  }
  const char* force = getenv("DWF_STAGE_VARIANT");
  int v = T.chosen >= 0 ? T.chosen : 0;
  if (force && force[0] >= '0' && force[0] < '0' + n && force[1] == 0) {
    v = force[0] - '0';
  } else if (T.chosen < 0 && T.next < nl && !capturing && a.stop == nullptr) {
    // launches that may return early (a solver's stop flag) are never timed: a converged
    // cycle would make the candidate that ran then look fast
    if (T.next == 0)
      for (int i = 0; i < 2 * nt; i++) cudaEventCreate(&T.ev[i]);
    v = T.next % n;
    const int j = T.next - n;   // timed launch index (the first round is not timed)
    if (j >= 0) cudaEventRecord(T.ev[2 * j], st);
    cudaError_t e = c[v].fn(b, c[v].smem, grid_of(c[v]), st);
    if (j >= 0) cudaEventRecord(T.ev[2 * j + 1], st);
    T.next++;
    T.pending = true;
    return e;
  }
  return c[v].fn(b, c[v].smem, grid_of(c[v]), st);
}

template <int P, int LS, bool DAG>
cudaError_t stage_dispatch_ls(const StageArgs& a, bool blocked, cudaStream_t st) {
  return blocked ? stage_launch_one<P, LS, DAG, true>(a, st)
                 : stage_launch_one<P, LS, DAG, false>(a, st);
}

}  // namespace dwf
