// The operator stage kernel: one launch computes, for every output site x of parity p and
// every slice s,
//
//   out(x,s) = hop_scale * [Post * Dh(in)](x,s) + [Loc * in2](x,s)
//
// where Dh is the Wilson hopping term (or its adjoint), Post is an optional dense
// per-chirality Ls x Ls matrix applied along the fifth dimension (D+ M5op^-1, M5op^-dag D+^dag,
// D+^dag), and Loc is the sparse M5op = alpha + beta K (or its adjoint).  Every piece of
//   Mpc    = M5op - 1/4 Dh_eo (D+ M5op^-1) Dh_oe D+,
//   Mpc^dag = M5op^dag - 1/4 D+^dag Dh^dag_eo (M5op^-dag D+^dag) Dh^dag_oe,
//   D      = M5op - 1/2 Dh D+,   D^dag = M5op^dag - 1/2 D+^dag Dh^dag
// is one such stage (Sec. 2.2 of the paper: DWF = Wilson hopping x fifth dimension).
//
// CTA = 32 consecutive sites x all Ls slices (thread (lane, s)).  The tile's links come from
// DRAM once and are reused by all Ls warps: copied into shared memory by TMA bulk copies, or
// prefetched into L2 and served from L1.  The Ls x Ls post (D+ M5op^-1 and its adjoint) runs
// over the CTA's 32 sites x 24 reals in shared memory: by bidiagonal recurrences, as a dense
// column GEMM, or on the tensor cores.  The epilogue optionally fuses the CG residual update
// r -= alpha * out and a deterministic ||.||^2 reduction.  Which variant runs is decided per
// stage kind by the launch autotuner (stage_inst.cuh).
#pragma once

#include "dwf_device.cuh"
#include "tc_m5.cuh"

namespace dwf {

enum LocalMode { LOC_NONE = 0, LOC_M5 = 1, LOC_M5DAG = 2 };
// EPI_NORM_ONLY: the reduction of EPI_NORM without storing the output (its only use)
enum EpiMode { EPI_STORE = 0, EPI_NORM = 1, EPI_CG_R = 2, EPI_NORM_ONLY = 3 };

struct StageArgs {
  const void* in;        // hop input, parity 1-p
  const void* in_halo;   // hop input for NBR_HALO neighbours (exact block operator)
  long Vp_in, Vp_halo;   // site strides of in / in_halo
  long Vp_link;          // site stride of the link array
  int skip_halo;         // treat NBR_HALO neighbours as absent
  void* out;             // output, parity p (EPI_STORE / EPI_NORM)
  const void* in2;       // local-term input, parity p (nullable if LOC_NONE)
  void* r;               // EPI_CG_R: residual updated in place
  const void* links;     // links of parity p: [8][9][Vp]
  const uint32_t* nbr;   // neighbours of parity p: [8][Vp]
  const void* post;      // [2][Ls][Ls] in the accumulation type, nullable
  const void* post_h;    // FP16/BF16 kernels: the same matrices as FP16 16x16 tensor-core
                         // operands (core-matrix layout); nullable = CUDA-core path
  int* err;              // set to 1 if a bounded device wait gives up (nullable)
  unsigned long long wait_ns;  // limit of every bounded device wait (0: the default 10 ms)
  int wait_probe;        // failure-detection test only: the TMA link staging issues no copy,
                         // so its wait runs out and the stage reports a timeout
  int post_sparse;       // the post matrix is D+^dag = dp_b + dp_c K^dag: apply it sparsely
  int post_struct;       // dense post D+ M5op^-1 (dag: M5op^-dag D+^dag) by O(Ls) recurrences:
                         // 0 no, 1 yes, 2 the faster of recurrences and tensor cores (16-bit)
  double dp_b, dp_c;
  double post_pre;       // extra factor of the structured post (b when the pre-op D+ = b)
  long Vp;               // site stride of out / in2 / r and of the neighbour table
  int Vhb, Vhb_pad;
  double hop_scale;
  int local_mode;
  double l_alpha, l_beta, mf;
  // filled from the fields above by finish_stage_args() at launch
  float hs32;
  Coef5<double> k64;
  Coef5<float> k32;
  int epi;
  const double* alpha;   // EPI_CG_R: per-segment alpha
  int seg_cps;           // CTAs per scalar/reduction segment (Vp/32: one global segment)
  const int* stop;       // nullable: skip everything when *stop != 0 (per segment if batched)
  RedArgs red;
  // batched mode (nullable): tile -> problem map and per-problem parameters; the problem's
  // post matrix is segp[seg].mat[post_which] when post is set
  const int* tile_seg;
  const BatchSeg* segp;
  int post_which;
  long ntiles;           // 32-site tiles (0: Vp / 32)
  int grid;              // CTAs of a persistent launch (0: one CTA per tile)
};

template <typename A>
__device__ __forceinline__ Coef5<A> coef5(const StageArgs& a) {
  if constexpr (sizeof(A) == 8) return a.k64; else return a.k32;
}
template <typename A>
__device__ __forceinline__ Coef5<A> coef5(const BatchSeg& S) {
  if constexpr (sizeof(A) == 8) return S.k64; else return S.k32;
}
inline void finish_stage_args(StageArgs& a, int Ls) {
  a.hs32 = (float)a.hop_scale;
  const double pre = a.post_pre != 0.0 ? a.post_pre : 1.0;
  a.k64 = make_coef5<double>(a.l_alpha, a.l_beta, a.mf, a.dp_b, a.dp_c, pre, Ls);
  a.k32 = make_coef5<float>(a.l_alpha, a.l_beta, a.mf, a.dp_b, a.dp_c, pre, Ls);
}

// 16-bit storage: the neighbour's spinor and the link stay packed in registers (12 + 12
// 32-bit words) and each element is converted to FP32 where it is used, which keeps the
// kernel's register footprint low enough for more resident CTAs per SM.
template <int P, int MU, bool SMEM = false>
__device__ __forceinline__ void hop_term16(Spinor<float>& acc, const uint4 (&q)[3],
                                           const uint4* lp, long Vl, float sgn) {
  constexpr bool BF = (P == PB16);
  const uint4 l0 = ldro<SMEM>(lp), l1 = ldro<SMEM>(lp + Vl), l2 = ldro<SMEM>(lp + 2 * Vl);
  auto sp = [&](int k) -> cx<float> {
    const uint4& w = q[k >> 2];
    const uint32_t v = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
    const float2 f = h2f(v, BF);
    return {f.x, f.y};
  };
  auto lk = [&](int k) -> cx<float> {
    const uint4& w = k < 4 ? l0 : (k < 8 ? l1 : l2);
    const uint32_t v = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
    const float2 f = h2f(v, BF);
    return {f.x, f.y};
  };
  cx<float> h[2][3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cx<float> p0 = sp(a), p1 = sp(3 + a), p2 = sp(6 + a), p3 = sp(9 + a);
    cx<float> b0, b1;
    if constexpr (MU == 0) {
      b0 = {p3.y, -p3.x};
      b1 = {p2.y, -p2.x};
    } else if constexpr (MU == 1) {
      b0 = {-p3.x, -p3.y};
      b1 = p2;
    } else if constexpr (MU == 2) {
      b0 = {p2.y, -p2.x};
      b1 = {-p3.y, p3.x};
    } else {
      b0 = p2;
      b1 = p3;
    }
    h[0][a] = {fmaf(sgn, b0.x, p0.x), fmaf(sgn, b0.y, p0.y)};
    h[1][a] = {fmaf(sgn, b1.x, p1.x), fmaf(sgn, b1.y, p1.y)};
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    cx<float> g0 = {0.f, 0.f}, g1 = {0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const cx<float> u = lk(a * 3 + b);
      cfma(g0, u, h[0][b]);
      cfma(g1, u, h[1][b]);
    }
    acc.c[a] = cadd(acc.c[a], g0);
    acc.c[3 + a] = cadd(acc.c[3 + a], g1);
    cx<float> l0, l1;   // B^dag g
    if constexpr (MU == 0) {
      l0 = {-g1.y, g1.x};
      l1 = {-g0.y, g0.x};
    } else if constexpr (MU == 1) {
      l0 = g1;
      l1 = {-g0.x, -g0.y};
    } else if constexpr (MU == 2) {
      l0 = {-g0.y, g0.x};
      l1 = {g1.y, -g1.x};
    } else {
      l0 = g0;
      l1 = g1;
    }
    acc.c[6 + a] = {fmaf(sgn, l0.x, acc.c[6 + a].x), fmaf(sgn, l0.y, acc.c[6 + a].y)};
    acc.c[9 + a] = {fmaf(sgn, l1.x, acc.c[9 + a].x), fmaf(sgn, l1.y, acc.c[9 + a].y)};
  }
}

// How a stage gathers the eight neighbour spinors and its links (a launch-variant choice, timed
// by the autotuner): neighbours straight into registers or through a two-slot cp.async ring in
// shared memory; links from global memory after an optional bulk L2 prefetch of the tile's
// links (G_BPF_L; G_BPF_LS / G_RING_BPF also prefetch the streamed inputs: local-term input,
// residual), or copied into shared memory by the TMA engine (G_TMA / G_RING_TMA: one
// cp.async.bulk per 512-byte run, completing on an mbarrier) and read by every warp from there.
// Either way each tile's links come from DRAM once and no direction waits on DRAM for them.
enum Gather { G_REG = 0, G_RING = 1, G_RING_BPF = 5, G_BPF_LS = 6, G_BPF_L = 7, G_TMA = 10,
              G_RING_TMA = 11 };
__host__ __device__ constexpr bool gather_ring(int g) {
  return g == G_RING || g == G_RING_BPF || g == G_RING_TMA;
}
__host__ __device__ constexpr bool gather_tma(int g) { return g == G_TMA || g == G_RING_TMA; }
// Slice mode of a stage launch: one fifth-dimension slice per thread, or two (slices w and
// w + Ls/2, each link read once for both; FP32 with the links in shared memory), the latter
// also with the two slices' components packed in float2 and f32x2 arithmetic.
enum SliceMode { SP_ONE = 1, SP_PAIR = 2, SP_PAIR_F2 = 3 };
__host__ __device__ constexpr int slices_per_thread(int sp) { return sp == SP_ONE ? 1 : 2; }
// bulk-prefetch depth of a gather mode: 0 none, 1 links, 2 links and streamed inputs
__host__ __device__ constexpr int bpf_what(int g) {
  return g == G_BPF_LS ? 2 : g == G_BPF_L ? 1 : g == G_RING_BPF ? 2 : 0;
}

__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(tc::smem_u32(mbar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy by the TMA engine; completes `bytes` on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar)) : "memory");
}

// Every run is 32 sites x 16 bytes = 512 bytes starting at the tile's first site (tiles cover
// [0, Vp)).  WHAT: 1 the tile's links, 2 also its streamed inputs (local-term input, residual).
// A bulk prefetch takes warp-uniform operands, so lane 0 of each warp issues its share (a
// per-lane loop would be serialised lane by lane).
template <int P, int LS, bool BLOCKED, int WHAT>
__device__ __forceinline__ void prefetch_tile(const StageArgs& a, long tile) {
  constexpr int NCH = Prec<P>::NCH, NCHL = Prec<P>::NCHL;
  constexpr int nrun = LS * NCH;   // (s, chunk) runs of one field
  const int warp = threadIdx.y, nw = blockDim.y;
  if (threadIdx.x != 0) return;
  const long base = tile * 32;
  const uint4* L = reinterpret_cast<const uint4*>(a.links);
  for (int i = warp; i < 8 * NCHL; i += nw) prefetch_l2_bulk(L + (long)i * a.Vp_link + base, 512);
  if constexpr (WHAT >= 2) {
    if (a.local_mode != LOC_NONE) {
      const uint4* Y = reinterpret_cast<const uint4*>(a.in2);
      for (int i = warp; i < nrun; i += nw) prefetch_l2_bulk(Y + (long)i * a.Vp + base, 512);
    }
    if (a.epi == EPI_CG_R) {
      const uint4* R = reinterpret_cast<const uint4*>(a.r);
      for (int i = warp; i < nrun; i += nw) prefetch_l2_bulk(R + (long)i * a.Vp + base, 512);
    }
  }
}

// source array, site stride and presence of the neighbour behind table entry nb
template <bool BLOCKED>
__device__ __forceinline__ bool nbr_source(const StageArgs& a, uint32_t nb, const void*& src,
                                           long& vs) {
  src = a.in;
  vs = a.Vp_in;
  if constexpr (BLOCKED) {
    if (nb & NBR_FACE) return false;
    if (nb & NBR_HALO) {
      if (a.skip_halo) return false;
      src = a.in_halo;
      vs = a.Vp_halo;
    }
  }
  return true;
}

// LSM: links from the tile's shared-memory copy lsm ([dir][chunk][32]; lsite = lane)
template <int P, int D, bool DAG, bool BLOCKED, bool LSM = false, bool COH = false>
__device__ __forceinline__ void hop_dir_nb(Spinor<typename Prec<P>::acc>& acc,
                                           const StageArgs& a, uint32_t nb, long lsite, int s,
                                           const void* lsm = nullptr) {
  using A = typename Prec<P>::acc;
  const void* src;
  long vs;
  if (!nbr_source<BLOCKED>(a, nb, src, vs)) return;
  const long j = (long)(nb & NBR_IDX);
  // forward hop: (1 - gamma_mu), backward: (1 + gamma_mu); the adjoint swaps them.
  constexpr bool back = (D & 1) != 0;
  const A sgn = (back != DAG) ? A(1) : A(-1);
  const void* lb = LSM ? lsm : a.links;
  const long vl = LSM ? 32 : a.Vp_link;
  if constexpr (P == P16 || P == PB16) {
    const uint4* p = reinterpret_cast<const uint4*>(src) + ((long)s * 3) * vs + j;
    const uint4 q[3] = {ldf<COH>(p), ldf<COH>(p + vs), ldf<COH>(p + 2 * vs)};
    const uint4* lp = reinterpret_cast<const uint4*>(lb) + (long)D * 3 * vl + lsite;
    hop_term16<P, D / 2, LSM>(acc, q, lp, vl, sgn);
  } else {
    Spinor<A> psi;
    load_spinor<P, COH>(psi, src, vs, j, s);
    hop_term<P, D / 2, LSM>(acc, psi, lb, vl, lsite, D, sgn);
  }
}

template <int P, int D, bool DAG, bool BLOCKED, bool LSM = false, bool COH = false>
__device__ __forceinline__ void hop_dir(Spinor<typename Prec<P>::acc>& acc, const StageArgs& a,
                                        long site, long lsite, int s,
                                        const void* lsm = nullptr) {
  hop_dir_nb<P, D, DAG, BLOCKED, LSM, COH>(acc, a, __ldg(a.nbr + (long)D * a.Vp + site), lsite,
                                           s, lsm);
}

// FP32 and 16-bit stages: the eight neighbour spinors are gathered with cp.async into a
// per-thread two-slot ring in shared memory, so the copy for direction d+1 is in flight while
// direction d is computed (each thread reads back only what it copied: no block barrier
// needed) and no registers are tied up by loads in flight.
template <bool L1>
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  if constexpr (L1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::
                     "r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))), "l"(gmem)
                 : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::
                     "r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// the gather ring lives at the start of dynamic shared memory: [2][NCH][32 Ls] x 16 bytes
template <int P>
__host__ __device__ constexpr size_t ring_bytes(int Ls) {
  return (P == P16 || P == PB16 || P == P32) ? (size_t)2 * Prec<P>::NCH * 32 * Ls * 16 : 0;
}

template <int P, bool DAG, bool BLOCKED, bool L1, bool LSM = false>
struct HopRing {
  static constexpr int NC = Prec<P>::NCH;
  const StageArgs& a;
  long site, lsite;
  int s, tid, nt;
  uint4* ring;          // [2][NC][nt] uint4
  const uint4* lsm;     // LSM: the tile's links in shared memory (lsite = lane)
  uint32_t nb[8];
  __device__ __forceinline__ bool present(int d) const {
    if constexpr (BLOCKED) {
      if (nb[d] & NBR_FACE) return false;
      if ((nb[d] & NBR_HALO) && a.skip_halo) return false;
    }
    return true;
  }
  __device__ __forceinline__ void issue(int d) {
    if (present(d)) {
      const void* src = a.in;
      long vs = a.Vp_in;
      if constexpr (BLOCKED) {
        if (nb[d] & NBR_HALO) {
          src = a.in_halo;
          vs = a.Vp_halo;
        }
      }
      const uint4* p =
          reinterpret_cast<const uint4*>(src) + ((long)s * NC) * vs + (nb[d] & NBR_IDX);
      uint4* slot = ring + (d & 1) * NC * nt + tid;
#pragma unroll
      for (int k = 0; k < NC; k++) cp_async16<L1>(slot + k * nt, p + k * vs);
    }
    cp_async_commit();
  }
  template <int D>
  __device__ __forceinline__ void compute(Spinor<float>& acc) {
    if (!present(D)) return;
    const uint4* slot = ring + (D & 1) * NC * nt + tid;
    constexpr bool back = (D & 1) != 0;
    const float sgn = (back != DAG) ? 1.f : -1.f;
    if constexpr (P == P32) {
      Spinor<float> psi;
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const float4 v = *reinterpret_cast<const float4*>(slot + k * nt);
        psi.c[2 * k] = {v.x, v.y};
        psi.c[2 * k + 1] = {v.z, v.w};
      }
      hop_term<P, D / 2>(acc, psi, a.links, a.Vp_link, lsite, D, sgn);
    } else {
      const uint4 q[3] = {slot[0], slot[nt], slot[2 * nt]};
      const long vl = LSM ? 32 : a.Vp_link;
      const uint4* lp = (LSM ? lsm : reinterpret_cast<const uint4*>(a.links)) + (long)D * 3 * vl +
                        lsite;
      hop_term16<P, D / 2, LSM>(acc, q, lp, vl, sgn);
    }
  }
  template <int D>
  __device__ __forceinline__ void step(Spinor<float>& acc) {
    if constexpr (D < 7) {
      issue(D + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    compute<D>(acc);
  }
  __device__ __forceinline__ void run(Spinor<float>& acc) {
#pragma unroll
    for (int d = 0; d < 8; d++) nb[d] = __ldg(a.nbr + (long)d * a.Vp + site);
    issue(0);
    step<0>(acc);
    step<1>(acc);
    step<2>(acc);
    step<3>(acc);
    step<4>(acc);
    step<5>(acc);
    step<6>(acc);
    step<7>(acc);
  }
};

// Dense per-chirality Ls x Ls matrix along s on the tensor cores (FP16/BF16 kernels): the
// CTA's 32 sites x 24 reals become A operands (rows = (real of one chirality, site), K = s'),
// six tcgen05 MMAs (M=128, N=16, K=16) accumulate in tensor memory, and the results come back
// through shared memory to the (site, s) threads.
//
// Shared memory of a tensor-core stage: [0, 3072 Ls) the 16-bit gather ring, reused for the
// staged results (both are exactly 3072 Ls bytes); then the six A tiles and the two B
// matrices.  The TMEM columns, the mbarrier, the B matrices and the zero K padding of the A
// tiles are set up once per CTA (tc_setup) and kept for every tile the CTA processes.
__host__ __device__ constexpr size_t tc_offset(int Ls) { return (size_t)3072 * Ls; }

template <int LS>
__device__ __forceinline__ void tc_setup(const StageArgs& a, unsigned char* smem,
                                         uint64_t* mbar, uint32_t* tslot) {
  constexpr int NT = 32 * LS;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  unsigned char* At = smem + tc_offset(LS);
  unsigned char* Bt = At + 6 * tc::TILE_BYTES;
  const uint4* bsrc = reinterpret_cast<const uint4*>(a.post_h);
  for (int i = tid; i < 2 * tc::B_BYTES / 16; i += NT) reinterpret_cast<uint4*>(Bt)[i] = bsrc[i];
  if constexpr (LS < 16) {
    constexpr int PADK = 16 - LS;
    for (int i = tid; i < 6 * 128 * PADK; i += NT) {
      const int j = i / (128 * PADK), rem = i % (128 * PADK);
      const int m = rem / PADK, k = LS + rem % PADK;
      *reinterpret_cast<__half*>(At + j * tc::TILE_BYTES + tc::core_offset(m, k)) =
          __float2half_rn(0.f);
    }
  }
  if (threadIdx.y == 0) tc::tmem_alloc(tslot, tc::TMEM_COLS);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// after the tile loop's final barrier: every tcgen05.ld has completed
__device__ __forceinline__ void tc_teardown(const uint32_t* tslot) {
  tc::fence_after_sync();
  if (threadIdx.y == 0) tc::tmem_dealloc(*tslot, tc::TMEM_COLS);
}

// Returns false (uniformly over the CTA) when the MMA completion wait gave up.
template <int LS>
__device__ __forceinline__ bool post_tensor_core(Spinor<float>& acc, const StageArgs& a,
                                                 int lane, int s, int tid,
                                                 unsigned char* smem, uint64_t* mbar,
                                                 uint32_t* tslot, uint32_t& phase) {
  unsigned char* At = smem + tc_offset(LS);
  const unsigned char* Bt = At + 6 * tc::TILE_BYTES;
  float* Dst = reinterpret_cast<float*>(smem);
#pragma unroll
  for (int c = 0; c < 24; c++) {
    const float v = (c & 1) ? acc.c[c >> 1].y : acc.c[c >> 1].x;
    const int chi = c / 12, cp = c % 12;
    const int f = cp * 32 + lane;
    const int j = chi * 3 + (f >> 7), m = f & 127;
    *reinterpret_cast<__half*>(At + j * tc::TILE_BYTES + tc::core_offset(m, s)) =
        __float2half_rn(v);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_f16(128, 16);
#pragma unroll
    for (int j = 0; j < 6; j++)
      tc::mma_f16(taddr + 16u * j, tc::smem_desc(tc::smem_u32(At + j * tc::TILE_BYTES)),
                  tc::smem_desc(tc::smem_u32(Bt + (j / 3) * tc::B_BYTES)), idesc, 0u);
    tc::mma_commit(mbar);
  }
  bool ok = tc::mbar_wait(mbar, phase, a.wait_ns);
  if (!ok) {
    // the MMAs may still be running: record the error, wait once more (bounded) for them
    if (a.err) atomicExch(a.err, 1);
    tc::mbar_wait(mbar, phase, a.wait_ns);
  }
  phase ^= 1u;
  tc::fence_after_sync();
  if (__syncthreads_or(!ok)) return false;
  // warp s reads the TMEM lane quarter q = s % 4 (rows 32q..32q+31 = real cp%4 = q of every
  // tile); the warps sharing a quarter split the six tiles between them.  The staging area is
  // the gather ring, idle since the barrier after the hop.
  const int q = s & 3;
  const int nq = (LS - q + 3) / 4;
  for (int j = s >> 2; j < 6; j += nq) {
    float v[16];
    tc::tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + 16u * j, v);
    const int chi = j / 3, cp = 4 * (j % 3) + q;
    const int c = 12 * chi + cp;
#pragma unroll
    for (int n = 0; n < LS; n++) Dst[(n * 24 + c) * 32 + lane] = v[n];
  }
  tc::fence_before_sync();
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 12; k++) {
    acc.c[k].x = Dst[(s * 24 + 2 * k) * 32 + lane];
    acc.c[k].y = Dst[(s * 24 + 2 * k + 1) * 32 + lane];
  }
  return true;
}

// Dynamic shared memory of a stage: the gather ring or the post matrices' staging area.
template <int P>
__host__ __device__ constexpr size_t stage_smem_base(int Ls, int post, int gather) {
  const size_t ring = gather_ring(gather) ? ring_bytes<P>(Ls) : 0;
  size_t need = 0;
  if (post == 1) need = (size_t)(Ls * 24 * 32 + 2 * Ls * Ls) * sizeof(typename Prec<P>::acc);
  if (post == 3 || post == 4) need = (size_t)Ls * 24 * 32 * sizeof(typename Prec<P>::acc);
  if (post == 2) need = tc_offset(Ls) + 6 * tc::TILE_BYTES + 2 * tc::B_BYTES;
  return need > ring ? need : ring;
}

// TMA link staging: the tile's 8 x NCHL link runs of 512 bytes after the ring / post area
template <int P>
__host__ __device__ constexpr size_t tma_link_offset(int Ls, int post, int gather) {
  return (stage_smem_base<P>(Ls, post, gather) + 127) / 128 * 128;
}
// POST: 0 = no post matrix, 1 = CUDA-core column GEMM, 2 = tensor cores (16-bit only),
//       3 = D+^dag applied sparsely (b + c K^dag: neighbours in s through shared memory),
//       4 = D+ M5op^-1 (dag: M5op^-dag D+^dag) by an O(Ls) recurrence per column
// One direction of the paired-slice hop: neighbour spinors of slices w and w + lsp, the link
// (from the tile's shared-memory copy) loaded once for both.
template <int P, int D, bool DAG, bool BLOCKED, bool COH = false>
__device__ __forceinline__ void hop_pair_d(Spinor<typename Prec<P>::acc> (&acc)[2],
                                           const StageArgs& a, long site, int lane, int w,
                                           int lsp, const uint4* lsm) {
  using A = typename Prec<P>::acc;
  const uint32_t nb = __ldg(a.nbr + (long)D * a.Vp + site);
  const void* src;
  long vs;
  if (!nbr_source<BLOCKED>(a, nb, src, vs)) return;
  const long j = (long)(nb & NBR_IDX);
  constexpr bool back = (D & 1) != 0;
  const A sgn = (back != DAG) ? A(1) : A(-1);
  Spinor<A> psi0, psi1;
  load_spinor<P, COH>(psi0, src, vs, j, w);
  load_spinor<P, COH>(psi1, src, vs, j, w + lsp);
  cx<A> u[9];
  load_link9<P, true>(u, lsm, 32, lane, D);
  hop_term_u<P, D / 2>(acc[0], psi0, u, sgn);
  hop_term_u<P, D / 2>(acc[1], psi1, u, sgn);
}

template <int P, bool DAG, bool BLOCKED, bool COH = false>
__device__ __forceinline__ void hop_pair(Spinor<typename Prec<P>::acc> (&acc)[2],
                                         const StageArgs& a, long site, int lane, int w,
                                         int lsp, const uint4* lsm) {
  hop_pair_d<P, 0, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 1, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 2, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 3, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 4, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 5, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 6, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_d<P, 7, DAG, BLOCKED, COH>(acc, a, site, lane, w, lsp, lsm);
}

// Packed paired-slice hop (FP32): component k of slices w and w + lsp shares one float2, so
// each f32x2 add or fma does the work of two FP32 instructions.  The projection to the
// half-spinor is done per slice (its results pair up in registers); the SU(3) products, with
// each link element broadcast to both halves, and the reconstruction run on the pairs.
struct cx2 {
  float2 x, y;   // real parts of the two slices, imaginary parts
};
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

template <int MU>
__device__ __forceinline__ void hop_term_f2(cx2 (&acc)[12], const Spinor<float>& psi0,
                                            const Spinor<float>& psi1, const cx<float> (&u)[9],
                                            float sgn) {
  cx<float> h0[2][3], h1[2][3];
  project_half<float, MU>(h0, psi0, sgn);
  project_half<float, MU>(h1, psi1, sgn);
  cx2 h[2][3];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      h[i][b] = {make_float2(h0[i][b].x, h1[i][b].x), make_float2(h0[i][b].y, h1[i][b].y)};
  const float2 m1 = bcast2(-1.f);
  cx2 g[2][3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const float2 ux0 = bcast2(u[3 * a].x), uy0 = bcast2(u[3 * a].y);
    const float2 ux1 = bcast2(u[3 * a + 1].x), uy1 = bcast2(u[3 * a + 1].y);
    const float2 ux2 = bcast2(u[3 * a + 2].x), uy2 = bcast2(u[3 * a + 2].y);
#pragma unroll
    for (int i = 0; i < 2; i++) {
      // re: sum u.x h.x - sum u.y h.y;  im: sum u.x h.y + sum u.y h.x
      float2 re = __fmul2_rn(ux0, h[i][0].x);
      re = __ffma2_rn(ux1, h[i][1].x, re);
      re = __ffma2_rn(ux2, h[i][2].x, re);
      float2 q = __fmul2_rn(uy0, h[i][0].y);
      q = __ffma2_rn(uy1, h[i][1].y, q);
      q = __ffma2_rn(uy2, h[i][2].y, q);
      float2 im = __fmul2_rn(ux0, h[i][0].y);
      im = __ffma2_rn(ux1, h[i][1].y, im);
      im = __ffma2_rn(ux2, h[i][2].y, im);
      im = __ffma2_rn(uy0, h[i][0].x, im);
      im = __ffma2_rn(uy1, h[i][1].x, im);
      im = __ffma2_rn(uy2, h[i][2].x, im);
      g[i][a] = {__ffma2_rn(q, m1, re), im};
    }
  }
  // acc += v (s > 0) or acc -= v (s < 0): multiplying by -1 is exact, so the fma rounds once
  // like a subtraction
  auto add = [&](float2& acc_, float2 v, bool neg) {
    acc_ = neg ? __ffma2_rn(v, m1, acc_) : __fadd2_rn(acc_, v);
  };
  const bool sn = sgn < 0.f;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    add(acc[a].x, g[0][a].x, false);
    add(acc[a].y, g[0][a].y, false);
    add(acc[3 + a].x, g[1][a].x, false);
    add(acc[3 + a].y, g[1][a].y, false);
    // lower spins: sgn * B^dag g, B^dag as in hop_term_u (i z = (-z.y, z.x))
    if constexpr (MU == 0) {          // l0 = i g1, l1 = i g0
      add(acc[6 + a].x, g[1][a].y, !sn);
      add(acc[6 + a].y, g[1][a].x, sn);
      add(acc[9 + a].x, g[0][a].y, !sn);
      add(acc[9 + a].y, g[0][a].x, sn);
    } else if constexpr (MU == 1) {   // l0 = g1, l1 = -g0
      add(acc[6 + a].x, g[1][a].x, sn);
      add(acc[6 + a].y, g[1][a].y, sn);
      add(acc[9 + a].x, g[0][a].x, !sn);
      add(acc[9 + a].y, g[0][a].y, !sn);
    } else if constexpr (MU == 2) {   // l0 = i g0, l1 = -i g1
      add(acc[6 + a].x, g[0][a].y, !sn);
      add(acc[6 + a].y, g[0][a].x, sn);
      add(acc[9 + a].x, g[1][a].y, sn);
      add(acc[9 + a].y, g[1][a].x, !sn);
    } else {                          // l0 = g0, l1 = g1
      add(acc[6 + a].x, g[0][a].x, sn);
      add(acc[6 + a].y, g[0][a].y, sn);
      add(acc[9 + a].x, g[1][a].x, sn);
      add(acc[9 + a].y, g[1][a].y, sn);
    }
  }
}

template <int D, bool DAG, bool BLOCKED>
__device__ __forceinline__ void hop_pair_f2_d(cx2 (&acc)[12], const StageArgs& a, long site,
                                              int lane, int w, int lsp, const uint4* lsm) {
  const uint32_t nb = __ldg(a.nbr + (long)D * a.Vp + site);
  const void* src;
  long vs;
  if (!nbr_source<BLOCKED>(a, nb, src, vs)) return;
  const long j = (long)(nb & NBR_IDX);
  constexpr bool back = (D & 1) != 0;
  constexpr float sgn = (back != DAG) ? 1.f : -1.f;
  Spinor<float> psi0, psi1;
  load_spinor<P32>(psi0, src, vs, j, w);
  load_spinor<P32>(psi1, src, vs, j, w + lsp);
  cx<float> u[9];
  load_link9<P32, true>(u, lsm, 32, lane, D);
  hop_term_f2<D / 2>(acc, psi0, psi1, u, sgn);
}

template <bool DAG, bool BLOCKED>
__device__ __forceinline__ void hop_pair_f2(Spinor<float> (&out)[2], const StageArgs& a,
                                            long site, int lane, int w, int lsp,
                                            const uint4* lsm) {
  cx2 acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  hop_pair_f2_d<0, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<1, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<2, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<3, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<4, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<5, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<6, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
  hop_pair_f2_d<7, DAG, BLOCKED>(acc, a, site, lane, w, lsp, lsm);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    out[0].c[k] = {acc[k].x.x, acc[k].y.x};
    out[1].c[k] = {acc[k].x.y, acc[k].y.y};
  }
}

// SP: slice mode (enum SliceMode).  In the paired modes thread (lane, w) computes slices w and
// w + Ls/2 and loads each link once for both.
// Returns false (uniformly over the CTA) when a bounded wait gave up: the caller stops.
template <int P, int LS, bool DAG, bool BLOCKED, int POST, int G, int SP = 1, bool COH = false>
__device__ __forceinline__ bool stage_tile(const StageArgs& a, long tile,
                                           unsigned char* smem_raw, double* red_scratch,
                                           uint64_t* tc_mbar, uint32_t* tc_slot,
                                           uint32_t& tc_phase, uint64_t* lk_mbar,
                                           uint32_t& lk_phase) {
  using A = typename Prec<P>::acc;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int tid = lane + 32 * w;
  constexpr int NSL = slices_per_thread(SP);
  constexpr int NT = 32 * LS / NSL;
  constexpr int LSP = LS / NSL;   // distance between a thread's slices
  const long site = tile * 32 + lane;
  int seg, ntl, jl, vh;
  long first;
  const void* post = a.post;
  if (a.tile_seg) {
    seg = __ldg(a.tile_seg + tile);
    const BatchSeg& S = a.segp[seg];
    if (a.stop && a.stop[seg]) return true;
    first = S.first_tile;
    ntl = S.ntiles;
    jl = (int)(tile - first) * 32 + lane;
    vh = S.Vh;
    if (POST) post = S.mat[a.post_which];
  } else {
    if (a.stop && *a.stop) return true;
    const int cps = a.Vhb_pad >> 5;
    seg = (int)(tile / a.seg_cps);
    first = (long)seg * a.seg_cps;
    ntl = a.seg_cps;
    jl = (int)(tile % cps) * 32 + lane;
    vh = a.Vhb;
  }
  const bool valid = jl < vh;
  // this tile's fifth-dimension coefficients (per problem when batched), read where used
  auto K5 = [&]() -> Coef5<A> { return a.tile_seg ? coef5<A>(a.segp[seg]) : coef5<A>(a); };

  Spinor<A> acc[NSL];
#pragma unroll
  for (int j = 0; j < NSL; j++) zero(acc[j]);
  // G_TMA / G_RING_TMA: stage the tile's links in shared memory (after the ring / post area)
  const uint4* lsm = nullptr;
  if constexpr (gather_tma(G)) {
    constexpr int NCHL = Prec<P>::NCHL;
    unsigned char* lk = smem_raw + tma_link_offset<P>(LS, POST, G);
    if (tid == 0 && !a.wait_probe) {
      tc::fence_proxy_async_smem();   // earlier generic reads of the buffer come first
      mbar_expect_tx(lk_mbar, 8 * NCHL * 512);
      const uint4* L = reinterpret_cast<const uint4*>(a.links);
      for (int i = 0; i < 8 * NCHL; i++)
        bulk_g2s(lk + i * 512, L + (long)i * a.Vp_link + tile * 32, 512, lk_mbar);
    }
    bool ok = tc::mbar_wait(lk_mbar, lk_phase, a.wait_ns);
    if (!ok) {
      // copies issued but not landed: record the error and wait once more (bounded) so that
      // none is in flight when the CTA leaves; with wait_probe nothing was issued
      if (a.err) atomicExch(a.err, 1);
      if (!a.wait_probe) tc::mbar_wait(lk_mbar, lk_phase, a.wait_ns);
    }
    lk_phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    lsm = reinterpret_cast<const uint4*>(lk);
  }
  if constexpr (SP == SP_ONE) {
    const int s = w;
    if constexpr (gather_ring(G)) {
      if constexpr (G == G_RING_BPF) prefetch_tile<P, LS, BLOCKED, 2>(a, tile);
      if (valid) {
        const long lsite = site;
        constexpr bool LSM = gather_tma(G);
        HopRing<P, DAG, BLOCKED, true, LSM> hp{
            a, site, LSM ? (long)lane : lsite, s, tid, NT, reinterpret_cast<uint4*>(smem_raw), lsm};
        hp.run(acc[0]);
      }
      // the post stage reuses shared memory that other threads' rings occupy
      __syncthreads();
    } else if (G == G_TMA) {
      if (valid) {
        hop_dir<P, 0, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 1, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 2, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 3, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 4, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 5, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 6, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
        hop_dir<P, 7, DAG, BLOCKED, true, COH>(acc[0], a, site, lane, s, lsm);
      }
    } else {
      if constexpr (bpf_what(G) > 0) prefetch_tile<P, LS, BLOCKED, bpf_what(G)>(a, tile);
      if (valid) {
        const long lsite = site;
        hop_dir<P, 0, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 1, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 2, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 3, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 4, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 5, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 6, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
        hop_dir<P, 7, DAG, BLOCKED, false, COH>(acc[0], a, site, lsite, s);
      }
    }
  } else {
    // paired slices (FP32, links staged in shared memory): one link load serves both slices
    static_assert(gather_tma(G), "paired slices read the links from shared memory");
    static_assert(SP != SP_PAIR_F2 || P == P32, "packed pairs are FP32 only");
    if (valid) {
      if constexpr (SP == SP_PAIR) hop_pair<P, DAG, BLOCKED, COH>(acc, a, site, lane, w, LSP, lsm);
      if constexpr (SP == SP_PAIR_F2) hop_pair_f2<DAG, BLOCKED>(acc, a, site, lane, w, LSP, lsm);
    }
  }

  if constexpr (POST == 2 && (P == P16 || P == PB16) && SP == SP_ONE) {
    if (!post_tensor_core<LS>(acc[0], a, lane, w, tid, smem_raw, tc_mbar, tc_slot, tc_phase))
      return false;
  }
  if constexpr (POST == 3) {
    // D+^dag h at s = b h_s + c (P+ h_{s+1} + P- h_{s-1}),  h_{Ls} = -mf h_0, h_{-1} = -mf h_{Ls-1}
    A* buf = reinterpret_cast<A*>(smem_raw);
#pragma unroll
    for (int j = 0; j < NSL; j++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        buf[((w + j * LSP) * 24 + 2 * k) * 32 + lane] = acc[j].c[k].x;
        buf[((w + j * LSP) * 24 + 2 * k + 1) * 32 + lane] = acc[j].c[k].y;
      }
    __syncthreads();
    const Coef5<A> C = K5();
    const A b_ = C.db, c_ = C.dc;
#pragma unroll
    for (int j = 0; j < NSL; j++) {
      const int s = w + j * LSP;
      const int su = s + 1 < LS ? s + 1 : 0, sd = s > 0 ? s - 1 : LS - 1;
      const A fu = (s + 1 < LS) ? A(1) : -C.mf, fd = (s > 0) ? A(1) : -C.mf;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const int sn = k < 6 ? su : sd;
        const A f = k < 6 ? fu : fd;
        acc[j].c[k].x = b_ * acc[j].c[k].x + c_ * f * buf[(sn * 24 + 2 * k) * 32 + lane];
        acc[j].c[k].y = b_ * acc[j].c[k].y + c_ * f * buf[(sn * 24 + 2 * k + 1) * 32 + lane];
      }
    }
  }
  if constexpr (POST == 4) {
    // Per chirality, K restricted to one chirality is a cyclic shift with a -mf corner:
    // lower (y_{s-1}) for P+ without dag and P- with dag, upper (y_{s+1}) otherwise.
    // M5op = alpha + beta K:  (I + r S) z = v with r = beta/alpha is solved by a one-sided
    // recurrence w and the Sherman-Morrison correction for the corner:
    //   lower: w_0 = v_0, w_s = v_s - r w_{s-1},  z_s = w_s + kappa (-r)^s w_{Ls-1},
    //   upper: mirror image, kappa = r mf / (1 + mf (-r)^Ls);  M5op^-1 v = z / alpha.
    A* buf = reinterpret_cast<A*>(smem_raw);
#pragma unroll
    for (int j = 0; j < NSL; j++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        buf[((w + j * LSP) * 24 + 2 * k) * 32 + lane] = acc[j].c[k].x;
        buf[((w + j * LSP) * 24 + 2 * k + 1) * 32 + lane] = acc[j].c[k].y;
      }
    __syncthreads();
    const Coef5<A> C = K5();
    const A r = C.r, inva = C.inva, kappa = C.kappa;
    const A b_ = C.db, c_ = C.dc, mfA = C.mf, pre = C.pre;
    for (int col = tid; col < 24 * 32; col += NT) {
      const int c = col >> 5, l = col & 31;
      const bool lower = ((c < 12) != DAG);
      A v[LS];
#pragma unroll
      for (int t = 0; t < LS; t++) v[t] = buf[(t * 24 + c) * 32 + l];
      if (DAG) {   // D+^dag first
        A u[LS];
#pragma unroll
        for (int t = 0; t < LS; t++) {
          const A nb = lower ? (t > 0 ? v[t - 1] : -mfA * v[LS - 1])
                             : (t + 1 < LS ? v[t + 1] : -mfA * v[0]);
          u[t] = b_ * v[t] + c_ * nb;
        }
#pragma unroll
        for (int t = 0; t < LS; t++) v[t] = u[t];
      }
      if (lower) {
#pragma unroll
        for (int t = 1; t < LS; t++) v[t] = v[t] - r * v[t - 1];
        const A e = kappa * v[LS - 1];
        A g = A(1);
#pragma unroll
        for (int t = 0; t < LS; t++) {
          v[t] = (v[t] + e * g) * inva;
          g *= -r;
        }
      } else {
#pragma unroll
        for (int t = LS - 2; t >= 0; t--) v[t] = v[t] - r * v[t + 1];
        const A e = kappa * v[0];
        A g = A(1);
#pragma unroll
        for (int t = LS - 1; t >= 0; t--) {
          v[t] = (v[t] + e * g) * inva;
          g *= -r;
        }
      }
      if (!DAG) {   // then D+ (times the absorbed pre-op factor)
        A u[LS];
#pragma unroll
        for (int t = 0; t < LS; t++) {
          const A nb = lower ? (t > 0 ? v[t - 1] : -mfA * v[LS - 1])
                             : (t + 1 < LS ? v[t + 1] : -mfA * v[0]);
          u[t] = pre * (b_ * v[t] + c_ * nb);
        }
#pragma unroll
        for (int t = 0; t < LS; t++) v[t] = u[t];
      }
#pragma unroll
      for (int t = 0; t < LS; t++) buf[(t * 24 + c) * 32 + l] = v[t];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NSL; j++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[j].c[k].x = buf[((w + j * LSP) * 24 + 2 * k) * 32 + lane];
        acc[j].c[k].y = buf[((w + j * LSP) * 24 + 2 * k + 1) * 32 + lane];
      }
  }
  if constexpr (POST == 1) {
    // Dense per-chirality Ls x Ls matrix along s: buf[s][24][32] holds the CTA's hop results;
    // each thread owns whole (component, site) columns and writes them back in place.
    A* buf = reinterpret_cast<A*>(smem_raw);
    A* mat = buf + LS * 24 * 32;
    const A* pm = reinterpret_cast<const A*>(post);
    for (int i = tid; i < 2 * LS * LS; i += NT) mat[i] = pm[i];
#pragma unroll
    for (int j = 0; j < NSL; j++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        buf[((w + j * LSP) * 24 + 2 * k) * 32 + lane] = acc[j].c[k].x;
        buf[((w + j * LSP) * 24 + 2 * k + 1) * 32 + lane] = acc[j].c[k].y;
      }
    __syncthreads();
    for (int col = tid; col < 24 * 32; col += NT) {
      const int c = col >> 5, l = col & 31;
      const A* m = mat + (c >= 12 ? LS * LS : 0);
      A v[LS];
#pragma unroll
      for (int t = 0; t < LS; t++) v[t] = buf[(t * 24 + c) * 32 + l];
#pragma unroll
      for (int u = 0; u < LS; u++) {
        A o = A(0);
#pragma unroll
        for (int t = 0; t < LS; t++) o = fma(m[u * LS + t], v[t], o);
        buf[(u * 24 + c) * 32 + l] = o;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NSL; j++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc[j].c[k].x = buf[((w + j * LSP) * 24 + 2 * k) * 32 + lane];
        acc[j].c[k].y = buf[((w + j * LSP) * 24 + 2 * k + 1) * 32 + lane];
      }
  }

  A nrm = A(0);   // this thread's share of the reduction, in the accumulation type
#pragma unroll
  for (int jj = 0; jj < NSL; jj++) {
    const int s = w + jj * LSP;
    Spinor<A>& acc_j = acc[jj];
    A hs;
    if constexpr (sizeof(A) == 8) hs = a.hop_scale; else hs = a.hs32;
  #pragma unroll
    for (int k = 0; k < 12; k++) acc_j.c[k] = cscale(hs, acc_j.c[k]);

    if (a.local_mode != LOC_NONE && valid) {
      // M5op x at s = alpha x_s + beta (P- x_{s+1} + P+ x_{s-1});
      // M5op^dag x at s = alpha x_s + beta (P+ x_{s+1} + P- x_{s-1});
      // x_{Ls} = -mf x_0, x_{-1} = -mf x_{Ls-1}.
      Spinor<A> x0, xu, xd;
      load_spinor<P, COH>(x0, a.in2, a.Vp, site, s);
      load_spinor<P, COH>(xu, a.in2, a.Vp, site, s + 1 < LS ? s + 1 : 0);
      load_spinor<P, COH>(xd, a.in2, a.Vp, site, s > 0 ? s - 1 : LS - 1);
      const Coef5<A> C = K5();
      const A fu = (s + 1 < LS) ? A(1) : -C.mf;
      const A fd = (s > 0) ? A(1) : -C.mf;
      const A la = C.la, lb = C.lb;
      const bool dagm = (a.local_mode == LOC_M5DAG);
  #pragma unroll
      for (int k = 0; k < 12; k++) {
        const bool plus = k < 6;
        const bool from_up = dagm ? plus : !plus;
        const cx<A> nb = from_up ? cscale(fu, xu.c[k]) : cscale(fd, xd.c[k]);
        acc_j.c[k].x += la * x0.c[k].x + lb * nb.x;
        acc_j.c[k].y += la * x0.c[k].y + lb * nb.y;
      }
    }

    if (a.epi == EPI_CG_R) {
      const A al = A(a.alpha[seg]);
      Spinor<A> rr;
      load_spinor<P, COH>(rr, a.r, a.Vp, site, s);
  #pragma unroll
      for (int k = 0; k < 12; k++) {
        rr.c[k].x -= al * acc_j.c[k].x;
        rr.c[k].y -= al * acc_j.c[k].y;
      }
      store_spinor<P>(a.r, a.Vp, site, s, rr);
      // the norm of what was stored (rounded to the storage precision)
      Spinor<A> back = rr;
      round_to_storage<P>(back);
      A part = A(0);   // per-thread partial in the accumulation type; FP64 across threads
  #pragma unroll
      for (int k = 0; k < 12; k++) part = fma(back.c[k].x, back.c[k].x, fma(back.c[k].y, back.c[k].y, part));
      nrm += part;
    } else {
      if (a.epi != EPI_NORM_ONLY) store_spinor<P>(a.out, a.Vp, site, s, acc_j);
      if (a.epi == EPI_NORM || a.epi == EPI_NORM_ONLY) {
        A part = A(0);
  #pragma unroll
        for (int k = 0; k < 12; k++) part = fma(acc_j.c[k].x, acc_j.c[k].x, fma(acc_j.c[k].y, acc_j.c[k].y, part));
        nrm += part;
      }
    }
  }
  if (a.epi != EPI_STORE) {
    A v[1] = {nrm};
    grid_reduce_seg<1, A>(a.red, v, red_scratch, tile, seg, first, ntl);
  }
  return true;
}

// MINB = resident CTAs per SM the register budget is sized for (2 or 3); the launcher's
// autotuner picks the faster one per kernel configuration.
// G: how the neighbours are gathered (enum Gather); SP: slice mode (enum SliceMode; block
// 32 x Ls / slices per thread).
template <int P, int LS, bool DAG, bool BLOCKED, int POST, int MINB, int G, int SP = 1>
__global__ void __launch_bounds__(32 * LS / slices_per_thread(SP), MINB) stage_kernel(const StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red_scratch[32];
  __shared__ uint64_t tc_mbar;
  __shared__ uint32_t tc_slot;
  constexpr bool TC = (POST == 2 && (P == P16 || P == PB16));
  if constexpr (TC) tc_setup<LS>(a, smem_raw, &tc_mbar, &tc_slot);
  __shared__ uint64_t lk_mbar;
  if constexpr (gather_tma(G)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) tc::mbar_init(&lk_mbar, 1);
    __syncthreads();
  }
  uint32_t tc_phase = 0, lk_phase = 0;
  for (long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    if (!stage_tile<P, LS, DAG, BLOCKED, POST, G, SP>(a, tile, smem_raw, red_scratch, &tc_mbar,
                                                      &tc_slot, tc_phase, &lk_mbar, lk_phase))
      break;
    __syncthreads();
  }
  if constexpr (TC) tc_teardown(&tc_slot);
}

template <int P>
size_t stage_smem_bytes(int Ls, int post, int gather) {
  if (gather_tma(gather))
    return tma_link_offset<P>(Ls, post, gather) + (size_t)8 * Prec<P>::NCHL * 512;
  return stage_smem_base<P>(Ls, post, gather);
}

}  // namespace dwf
