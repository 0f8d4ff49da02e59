// The multisplitting preconditioner's local solves (Sec. 2.3, Eqs. 4-5) in one persistent,
// cooperative kernel: l iterations of plain CG on A_s x_s = r_s for every lattice block s at
// once, zero initial guess, block-local dot products.
//
// Block-SIMD layout.  All blocks have the same shape, so the sites a block's operator touches
// are the same set of block-relative positions for every block: BE/BO (the block's even/odd
// sites), and for A_s = P_s A P_s also HO (odd sites one hop outside, where D_oe of a
// block-supported vector lives) and HE (even sites outside reached from BO or HO, where Mpc of
// a block-supported vector lives).  E = BE ++ HE and O = BO ++ HO are stored position-major:
// element e = position * NB + block, so the 32 lanes of a warp are 32 blocks at one position.
// Every lane then has the same neighbour pattern (one broadcast table entry per direction, no
// divergence, hops that are absent at that position skipped as a whole), and every neighbour
// load is 32 consecutive elements of a 16-byte chunk (512 contiguous bytes).  Each block owns
// its halo positions, so blocks never exchange data: the local solves need no communication,
// as in the paper.
//
// Work split.  Blocks come in groups of 32 (one lane each); a fixed set of C CTAs (a "slot")
// runs every phase of every iteration of its block groups, each CTA taking positions from a
// cost-sorted schedule in round robin.  A CTA is 32 lanes x Ls/NSL warps; each thread handles
// NSL fifth-dimension slices (two for FP32/FP16/BF16: slices w and w + Ls/2 share every link
// load and run the SU(3) products in packed f32x2 arithmetic; one for FP64).  Phases of one CG
// iteration on A_s = Mpc_s^dag Mpc_s:
//   P1  t = [D+ M5op^-1] Dh_oe (D+ p)        on O  (input on BE)
//   P2  y = M5op p - 1/4 Dh_eo t             on E, per-block ||y||^2 = <p, A_s p> -> alpha
//   P3  s = [M5op^-dag D+^dag] Dh_oe^dag y   on O
//   P4  r -= alpha (M5op^dag y - 1/4 D+^dag Dh_eo^dag s)  on BE, per-block ||r||^2 -> beta
//   P5  x += alpha p, p = r + beta p, u = D+ p            on BE
// separated by barriers among the slot's CTAs only (a counter in global memory; every wait
// is bounded in time and reports an error instead of hanging).  The per-block reductions are
// one FP64 partial per (CTA, block), summed in a fixed order by every CTA after the barrier
// (deterministic, and every CTA holds the same alpha and beta).  The launch is cooperative, so
// all CTAs are resident at once.
#pragma once

#include <type_traits>

#include "dwf_device.cuh"
#include "stage.cuh"
#include "sync.cuh"
#include "tc_m5.cuh"

namespace dwf {

constexpr uint32_t SIMD_ABSENT = 0xffffffffu;

struct SimdArgs {
  int NB, nb, nBE, nE, nO;       // block stride, blocks, positions of BE / E / O
  int ngroups, C, nslots;        // 32-block groups, CTAs per slot, slots
  long sB, sE, sO;               // element strides of BE, E and O fields (positions * NB)
  const uint32_t* nbrE;          // [nE][8]: neighbour position in O, or SIMD_ABSENT
  const uint32_t* nbrO;          // [nO][8]: neighbour position in E, or SIMD_ABSENT
  const uint32_t* sch[4];        // cost-sorted entries of P1 (O), P2 (E), P3 (O), P4 (BE):
                                 // position | live-hop mask << 24
  int nsch[4];
  const void* linksE;            // [8][NCHL][sE] links of the E sites (backward ones daggered)
  const void* linksO;            // [8][NCHL][sO]
  const int* fwd;                // [sB]: BE element -> site of the outer field (-1: none)
  void *x, *p, *u, *r;           // BE fields
  void* t;                       // O field (t, then s)
  void* y;                       // E field
  const void* r_outer;           // residual of the outer iteration, [s][chunk][Vp_outer]
  int prec_outer;
  long Vp_outer;
  double num;                    // r_local = f r_outer, f = sqrt(num / *den) or num (den null)
  const double* den;
  Coef5<double> k64;             // M5op = la + lb K, D+ = db + dc K, recurrence r, inva, kappa,
  Coef5<float> k32;              // pre = b when D+ = b (absorbed pre-op), else 1
  double hs_b;                   // hop scale of the last stage: -1/4, or -b/4 when D+ = b
  int trivial;                   // c == 0: D+ = b, no pre-op field u
  int l;                         // local iterations
  int ncol, col;                 // Schwarz sweeps: only blocks of colour col (of ncol) solve;
                                 // the others get r = 0 and so x = 0 (ncol = 1: every block)
  int nbk[4];                    // blocks per direction (block b = b_x + nbk_x (b_y + ...))
  unsigned* ctr;                 // [nslots] barrier counters, zero at launch
  double* partial;               // [nslots][C][32] per-CTA, per-block partial sums
  unsigned long long wait_ns;
  int* err;
};

template <typename A>
__device__ __forceinline__ Coef5<A> simd_coef(const SimdArgs& a) {
  if constexpr (sizeof(A) == 8) return a.k64; else return a.k32;
}

// slices per thread
template <int P>
__host__ __device__ constexpr int simd_nsl() { return P == P64 ? 1 : 2; }

// Spinor of element e, slice s, from a field written earlier in this kernel (loads through
// L2: another SM may have written it since this SM last cached the line).
template <int P>
__device__ __forceinline__ void ld_spinor(Spinor<typename Prec<P>::acc>& out, const void* base,
                                          long stride, long e, int s) {
  constexpr int NCH = Prec<P>::NCH;
  const uint4* q = reinterpret_cast<const uint4*>(base) + ((long)s * NCH) * stride + e;
  if constexpr (P == P64) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(q + k * stride));
      out.c[k] = {v.x, v.y};
    }
  } else if constexpr (P == P32) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(q + k * stride));
      out.c[2 * k] = {v.x, v.y};
      out.c[2 * k + 1] = {v.z, v.w};
    }
  } else {
    constexpr bool BF = (P == PB16);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint4 v = __ldcg(q + k * stride);
      const float2 a = h2f(v.x, BF), b = h2f(v.y, BF), c = h2f(v.z, BF), d = h2f(v.w, BF);
      out.c[4 * k] = {a.x, a.y};
      out.c[4 * k + 1] = {b.x, b.y};
      out.c[4 * k + 2] = {c.x, c.y};
      out.c[4 * k + 3] = {d.x, d.y};
    }
  }
}

// Shared memory of the local-solve kernel: two buffers of raw tile links ([8][NCHL][32] chunks
// of 16 bytes; the next tile's links are copied in while the current tile computes), then one
// region used first as the per-thread neighbour ring ([2][NSL][NCH][threads] chunks; not for
// FP64, which loads neighbours directly) and then as the fifth-dimension buffer ([LS][24][32]).
template <int P>
__host__ __device__ constexpr size_t simd_lraw_bytes() {
  return (size_t)8 * Prec<P>::NCHL * 32 * 16;
}
template <int P>
__host__ __device__ constexpr bool simd_ring() { return P != P64; }
template <int P>
__host__ __device__ constexpr size_t simd_region_bytes(int ls, int rs) {
  const size_t ring = simd_ring<P>() ? (size_t)rs * Prec<P>::NCH * 32 * ls * 16 : 0;
  const size_t buf = (size_t)ls * 24 * 32 * sizeof(typename Prec<P>::acc);
  return ring > buf ? ring : buf;
}
template <int P>
__host__ __device__ constexpr size_t simd_smem_bytes(int ls, int rs) {
  return 2 * simd_lraw_bytes<P>() + simd_region_bytes<P>(ls, rs);
}

// Copies the links of the live directions of the tile at element e0 into lraw (cp.async
// through L2; one commit group per thread).
template <int P>
__device__ __forceinline__ void simd_prefetch_links(uint4* lraw, const void* links, long stride,
                                                    long e0, uint32_t live, int tid, int nt) {
  constexpr int NCHL = Prec<P>::NCHL;
  const uint4* L = reinterpret_cast<const uint4*>(links);
  for (int i = tid; i < 8 * NCHL * 32; i += nt) {
    const int d = i / (NCHL * 32);
    if (!((live >> d) & 1u)) continue;
    const int ch = (i >> 5) % NCHL, ln = i & 31;
    cp_async16<false>(lraw + i, L + (long)(d * NCHL + ch) * stride + e0 + ln);
  }
  cp_async_commit();
}

// Schedule entry: the position in the low 24 bits, the mask of its live hops above.
constexpr uint32_t SIMD_POS_MASK = 0x00ffffffu;

// The spinor of NCH 16-byte chunks q[0], q[qs], ... in the accumulation type.
template <int P>
__device__ __forceinline__ void unpack_chunks(Spinor<typename Prec<P>::acc>& psi, const uint4* q,
                                              int qs) {
  if constexpr (P == P64) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 v = *reinterpret_cast<const double2*>(q + k * qs);
      psi.c[k] = {v.x, v.y};
    }
  } else if constexpr (P == P32) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 v = *reinterpret_cast<const float4*>(q + k * qs);
      psi.c[2 * k] = {v.x, v.y};
      psi.c[2 * k + 1] = {v.z, v.w};
    }
  } else {
    constexpr bool BF = (P == PB16);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint4 v = q[k * qs];
      const float2 a = h2f(v.x, BF), b = h2f(v.y, BF), c = h2f(v.z, BF), d = h2f(v.w, BF);
      psi.c[4 * k] = {a.x, a.y};
      psi.c[4 * k + 1] = {b.x, b.y};
      psi.c[4 * k + 2] = {c.x, c.y};
      psi.c[4 * k + 3] = {d.x, d.y};
    }
  }
}

// Accumulator of a thread's NSL slices: FP64 one Spinor, the others packed pairs (cx2: the
// two slices' components side by side in float2 registers).
template <int P>
struct HopAcc {
  cx2 c[12];
};
template <>
struct HopAcc<P64> {
  Spinor<double> s;
};

template <int P>
__device__ __forceinline__ void hop_acc_zero(HopAcc<P>& h) {
  if constexpr (P == P64) {
    zero(h.s);
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) h.c[k] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  }
}
template <int P, int NSL>
__device__ __forceinline__ void hop_acc_out(const HopAcc<P>& h,
                                            Spinor<typename Prec<P>::acc> (&out)[NSL]) {
  if constexpr (P == P64) {
    out[0] = h.s;
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      out[0].c[k] = {h.c[k].x.x, h.c[k].y.x};
      out[1].c[k] = {h.c[k].x.y, h.c[k].y.y};
    }
  }
}

// One hop direction D for the thread's slices: spinors from the chunks at q (slice j at
// q + j * jstride, chunk k at + k * qs), the link from the tile's raw copy.
template <int P, bool DAG, int D>
__device__ __forceinline__ void simd_term(HopAcc<P>& acc, const uint4* q, int qs, int jstride,
                                          const uint4* lraw, int lane) {
  using A = typename Prec<P>::acc;
  constexpr bool back = (D & 1) != 0;
  const A sgn = (back != DAG) ? A(1) : A(-1);
  cx<A> u[9];
  load_link9<P, true>(u, lraw, 32, lane, D);
  if constexpr (P == P64) {
    Spinor<A> psi;
    unpack_chunks<P>(psi, q, qs);
    hop_term_u<P, D / 2>(acc.s, psi, u, sgn);
  } else {
    Spinor<float> psi0, psi1;
    unpack_chunks<P>(psi0, q, qs);
    unpack_chunks<P>(psi1, q + jstride, qs);
    hop_term_f2<D / 2>(acc.c, psi0, psi1, u, sgn);
  }
}

template <int P, bool DAG>
__device__ __forceinline__ void simd_term_d(int d, HopAcc<P>& acc, const uint4* q, int qs,
                                            int jstride, const uint4* lraw, int lane) {
  switch (d) {
    case 0: simd_term<P, DAG, 0>(acc, q, qs, jstride, lraw, lane); break;
    case 1: simd_term<P, DAG, 1>(acc, q, qs, jstride, lraw, lane); break;
    case 2: simd_term<P, DAG, 2>(acc, q, qs, jstride, lraw, lane); break;
    case 3: simd_term<P, DAG, 3>(acc, q, qs, jstride, lraw, lane); break;
    case 4: simd_term<P, DAG, 4>(acc, q, qs, jstride, lraw, lane); break;
    case 5: simd_term<P, DAG, 5>(acc, q, qs, jstride, lraw, lane); break;
    case 6: simd_term<P, DAG, 6>(acc, q, qs, jstride, lraw, lane); break;
    default: simd_term<P, DAG, 7>(acc, q, qs, jstride, lraw, lane); break;
  }
}

// acc += sum over the live directions of the hop from `in` (element nb * NB + eg) for the
// thread's slices w (+ LS/2), with the tile's links in lraw.  16-bit and FP32: the neighbour
// spinors go through a two-slot cp.async ring in shared memory, so the copy of the next live
// direction is in flight while the current one is computed (each thread reads back only its
// own copies: no block barrier).
template <int P, int LS, bool DAG, int RS>
__device__ __forceinline__ void simd_hop(HopAcc<P>& acc, const uint32_t* row, uint32_t live,
                                         const void* in, long stride, int NB, long eg, int w,
                                         const uint4* lraw, uint4* ring, int lane, int tid) {
  constexpr int NCH = Prec<P>::NCH;
  constexpr int NSL = simd_nsl<P>();
  constexpr int LSP = LS / NSL;
  constexpr int NT = 32 * LSP;
  if constexpr (!simd_ring<P>()) {
#pragma unroll
    for (int d = 0; d < 8; d++) {
      if (!((live >> d) & 1u)) continue;
      const uint4* q = reinterpret_cast<const uint4*>(in) + ((long)w * NCH) * stride +
                       (long)row[d] * NB + eg;
      uint4 v[NCH];
#pragma unroll
      for (int k = 0; k < NCH; k++) v[k] = __ldcg(q + k * stride);
      simd_term_d<P, DAG>(d, acc, v, 1, 0, lraw, lane);
    }
  } else {
    // ring slot layout: [slot][slice j][chunk k][thread]; RS slots keep RS - 1 directions in
    // flight ahead of the one being computed
    auto issue = [&](int d, int slot) {
      const uint4* q = reinterpret_cast<const uint4*>(in) + ((long)w * NCH) * stride +
                       (long)row[d] * NB + eg;
      uint4* dst = ring + (slot * NSL * NCH) * NT + tid;
#pragma unroll
      for (int j = 0; j < NSL; j++)
#pragma unroll
        for (int k = 0; k < NCH; k++)
          cp_async16<false>(dst + (j * NCH + k) * NT, q + ((long)j * LSP * NCH + k) * stride);
      cp_async_commit();
    };
    // the i-th live direction (i from 0): clear the i lowest set bits
    auto nth = [&](int i) {
      uint32_t m = live;
      for (int k = 0; k < i; k++) m &= m - 1u;
      return __ffs(m) - 1;
    };
    const int n = __popc(live);
#pragma unroll
    for (int i = 0; i < RS - 1; i++)
      if (i < n) issue(nth(i), i);
    for (int i = 0; i < n; i++) {
      if (i + RS - 1 < n) issue(nth(i + RS - 1), (i + RS - 1) % RS);
      const int newer = min(RS - 1, n - 1 - i);   // groups committed after direction i's
      if (newer >= 2) cp_async_wait<2>();
      else if (newer == 1) cp_async_wait<1>();
      else cp_async_wait<0>();
      const uint4* q = ring + ((i % RS) * NSL * NCH) * NT + tid;
      simd_term_d<P, DAG>(nth(i), acc, q, NT, NCH * NT, lraw, lane);
    }
  }
}

// The hop of the tile, unpacked into one spinor per slice of the thread.
template <int P, int LS, bool DAG, int RS>
__device__ __forceinline__ void simd_hop_out(Spinor<typename Prec<P>::acc> (&out)[simd_nsl<P>()],
                                             const uint32_t* row, uint32_t live, const void* in,
                                             long stride, int NB, long eg, int w,
                                             const uint4* lraw, uint4* ring, int lane, int tid) {
  HopAcc<P> h;
  hop_acc_zero<P>(h);
  simd_hop<P, LS, DAG, RS>(h, row, live, in, stride, NB, eg, w, lraw, ring, lane, tid);
  hop_acc_out<P, simd_nsl<P>()>(h, out);
}

// The fifth-dimension buffer <-> the per-thread spinor of slice s.  FP32 accumulation: float4
// quads, buf[(s * 6 + q) * 32 + lane] = components 2q, 2q + 1 (re, im, re, im), so a warp moves
// 512 contiguous bytes per quad; FP64: scalars, buf[(s * 24 + k) * 32 + lane].
template <typename A>
__device__ __forceinline__ void to_buf(A* buf, const Spinor<A>& v, int s, int lane) {
  if constexpr (std::is_same<A, float>::value) {
    float4* b4 = reinterpret_cast<float4*>(buf);
#pragma unroll
    for (int q = 0; q < 6; q++)
      b4[(s * 6 + q) * 32 + lane] =
          make_float4(v.c[2 * q].x, v.c[2 * q].y, v.c[2 * q + 1].x, v.c[2 * q + 1].y);
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      buf[(s * 24 + 2 * k) * 32 + lane] = v.c[k].x;
      buf[(s * 24 + 2 * k + 1) * 32 + lane] = v.c[k].y;
    }
  }
}
template <typename A>
__device__ __forceinline__ void from_buf(Spinor<A>& v, const A* buf, int s, int lane) {
  if constexpr (std::is_same<A, float>::value) {
    const float4* b4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const float4 t = b4[(s * 6 + q) * 32 + lane];
      v.c[2 * q] = {t.x, t.y};
      v.c[2 * q + 1] = {t.z, t.w};
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      v.c[k].x = buf[(s * 24 + 2 * k) * 32 + lane];
      v.c[k].y = buf[(s * 24 + 2 * k + 1) * 32 + lane];
    }
  }
}

// Fifth-dimension post on the CTA's 32 x 24 columns in buf: D+ M5op^-1 (DAG false, times the
// absorbed pre-op factor) or M5op^-dag D+^dag (DAG true).  Per chirality K is a cyclic shift
// with a -mf corner, so M5op = la (1 + r S) is inverted by a one-sided recurrence plus the
// Sherman-Morrison correction for the corner, kappa = r mf / (1 + mf (-r)^Ls).
// FP32 accumulation: one work item is a quad of four columns of one chirality (q < 3: the
// upper spins), run as two packed f32x2 column pairs; FP64: one column per item.
template <int LS, bool DAG>
__device__ __forceinline__ void post_recurrence_q(float* bufp, const Coef5<float>& C, int tid,
                                                  int nt) {
  float4* buf = reinterpret_cast<float4*>(bufp);
  const float2 mr = bcast2(-C.r), inva = bcast2(C.inva);
  const float2 b2 = bcast2(DAG ? C.db : C.pre * C.db), c2 = bcast2(DAG ? C.dc : C.pre * C.dc);
  const float2 cw = bcast2(-C.mf * (DAG ? C.dc : C.pre * C.dc));   // the wall term's factor
  for (int it = tid; it < 6 * 32; it += nt) {
    const int q = it >> 5, l = it & 31;
    const bool lower = ((q < 3) != DAG);
    float2 v[LS][2];
#pragma unroll
    for (int t = 0; t < LS; t++) {
      const float4 x = buf[(t * 6 + q) * 32 + l];
      v[t][0] = make_float2(x.x, x.y);
      v[t][1] = make_float2(x.z, x.w);
    }
    // D+ (or D+^dag) in place: w_t = b v_t + c v_{t-1} (lower; the wall: -mf v_{Ls-1}) or
    // w_t = b v_t + c v_{t+1} (upper; the wall: -mf v_0)
    auto dplus = [&](float2 (&vv)[LS][2], float2 bb, float2 cc, float2 cwall) {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (lower) {
          const float2 wrap = vv[LS - 1][h];
#pragma unroll
          for (int t = LS - 1; t > 0; t--) vv[t][h] = __ffma2_rn(cc, vv[t - 1][h], __fmul2_rn(bb, vv[t][h]));
          vv[0][h] = __ffma2_rn(cwall, wrap, __fmul2_rn(bb, vv[0][h]));
        } else {
          const float2 wrap = vv[0][h];
#pragma unroll
          for (int t = 0; t + 1 < LS; t++) vv[t][h] = __ffma2_rn(cc, vv[t + 1][h], __fmul2_rn(bb, vv[t][h]));
          vv[LS - 1][h] = __ffma2_rn(cwall, wrap, __fmul2_rn(bb, vv[LS - 1][h]));
        }
      }
    };
    if (DAG) dplus(v, b2, c2, cw);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (lower) {
#pragma unroll
        for (int t = 1; t < LS; t++) v[t][h] = __ffma2_rn(mr, v[t - 1][h], v[t][h]);
        const float2 e = __fmul2_rn(bcast2(C.kappa), v[LS - 1][h]);
        float g = 1.f;
#pragma unroll
        for (int t = 0; t < LS; t++) {
          v[t][h] = __fmul2_rn(__ffma2_rn(e, bcast2(g), v[t][h]), inva);
          g *= -C.r;
        }
      } else {
#pragma unroll
        for (int t = LS - 2; t >= 0; t--) v[t][h] = __ffma2_rn(mr, v[t + 1][h], v[t][h]);
        const float2 e = __fmul2_rn(bcast2(C.kappa), v[0][h]);
        float g = 1.f;
#pragma unroll
        for (int t = LS - 1; t >= 0; t--) {
          v[t][h] = __fmul2_rn(__ffma2_rn(e, bcast2(g), v[t][h]), inva);
          g *= -C.r;
        }
      }
    }
    if (!DAG) dplus(v, b2, c2, cw);
#pragma unroll
    for (int t = 0; t < LS; t++)
      buf[(t * 6 + q) * 32 + l] = make_float4(v[t][0].x, v[t][0].y, v[t][1].x, v[t][1].y);
  }
}

template <typename A, int LS, bool DAG>
__device__ __forceinline__ void post_recurrence(A* buf, const Coef5<A>& C, int tid, int nt) {
  if constexpr (std::is_same<A, float>::value) {
    post_recurrence_q<LS, DAG>(buf, C, tid, nt);
    return;
  } else {
    const A r = C.r, inva = C.inva, kappa = C.kappa;
    const A b_ = C.db, c_ = C.dc, mfA = C.mf, pre = C.pre;
    for (int col = tid; col < 24 * 32; col += nt) {
      const int c = col >> 5, l = col & 31;
      const bool lower = ((c < 12) != DAG);
      A v[LS];
#pragma unroll
      for (int t = 0; t < LS; t++) v[t] = buf[(t * 24 + c) * 32 + l];
      if (DAG) {   // D+^dag first
        A w[LS];
#pragma unroll
        for (int t = 0; t < LS; t++) {
          const A nb = lower ? (t > 0 ? v[t - 1] : -mfA * v[LS - 1])
                             : (t + 1 < LS ? v[t + 1] : -mfA * v[0]);
          w[t] = b_ * v[t] + c_ * nb;
        }
#pragma unroll
        for (int t = 0; t < LS; t++) v[t] = w[t];
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
        A w[LS];
#pragma unroll
        for (int t = 0; t < LS; t++) {
          const A nb = lower ? (t > 0 ? v[t - 1] : -mfA * v[LS - 1])
                             : (t + 1 < LS ? v[t + 1] : -mfA * v[0]);
          w[t] = pre * (b_ * v[t] + c_ * nb);
        }
#pragma unroll
        for (int t = 0; t < LS; t++) v[t] = w[t];
      }
#pragma unroll
      for (int t = 0; t < LS; t++) buf[(t * 24 + c) * 32 + l] = v[t];
    }
  }
}

// v[j] <- D+ v[j] (P+ spins from s-1, P- spins from s+1, -mf at the walls), or D+^dag (P+ from
// s+1, P- from s-1), for the thread's slices s_j = w + j LS/NSL, through buf (filled here).
template <typename A, int LS, int NSL, bool DAG>
__device__ __forceinline__ void dplus_slices(Spinor<A> (&v)[NSL], A* buf, const Coef5<A>& C,
                                             int w, int lane) {
  constexpr int LSP = LS / NSL;
#pragma unroll
  for (int j = 0; j < NSL; j++) to_buf(buf, v[j], w + j * LSP, lane);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NSL; j++) {
    const int s = w + j * LSP;
    const int su = s + 1 < LS ? s + 1 : 0, sd = s > 0 ? s - 1 : LS - 1;
    const A fu = (s + 1 < LS) ? A(1) : -C.mf, fd = (s > 0) ? A(1) : -C.mf;
    if constexpr (std::is_same<A, float>::value) {
      const float4* b4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
      for (int q = 0; q < 6; q++) {   // components 2q, 2q + 1: P+ spins for q < 3
        const bool from_up = DAG ? (q < 3) : (q >= 3);
        const float4 t = b4[((from_up ? su : sd) * 6 + q) * 32 + lane];
        const float f = C.dc * (from_up ? fu : fd);
        v[j].c[2 * q].x = C.db * v[j].c[2 * q].x + f * t.x;
        v[j].c[2 * q].y = C.db * v[j].c[2 * q].y + f * t.y;
        v[j].c[2 * q + 1].x = C.db * v[j].c[2 * q + 1].x + f * t.z;
        v[j].c[2 * q + 1].y = C.db * v[j].c[2 * q + 1].y + f * t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) {
        const bool plus = k < 6;
        const bool from_up = DAG ? plus : !plus;
        const int sn = from_up ? su : sd;
        const A f = from_up ? fu : fd;
        v[j].c[k].x = C.db * v[j].c[k].x + C.dc * f * buf[(sn * 24 + 2 * k) * 32 + lane];
        v[j].c[k].y = C.db * v[j].c[k].y + C.dc * f * buf[(sn * 24 + 2 * k + 1) * 32 + lane];
      }
    }
  }
  __syncthreads();
}

// acc += M5op x (DAG false) or M5op^dag x (DAG true) at slice s: la x_s + lb (K or K^dag) x.
template <int P, bool DAG>
__device__ __forceinline__ void add_m5(Spinor<typename Prec<P>::acc>& acc, const void* x,
                                       long stride, long e, int s, int ls,
                                       const Coef5<typename Prec<P>::acc>& C) {
  using A = typename Prec<P>::acc;
  Spinor<A> x0, xu, xd;
  ld_spinor<P>(x0, x, stride, e, s);
  ld_spinor<P>(xu, x, stride, e, s + 1 < ls ? s + 1 : 0);
  ld_spinor<P>(xd, x, stride, e, s > 0 ? s - 1 : ls - 1);
  const A fu = (s + 1 < ls) ? A(1) : -C.mf, fd = (s > 0) ? A(1) : -C.mf;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const bool plus = k < 6;
    const bool from_up = DAG ? plus : !plus;
    const cx<A> nb = from_up ? cscale(fu, xu.c[k]) : cscale(fd, xd.c[k]);
    acc.c[k].x += C.la * x0.c[k].x + C.lb * nb.x;
    acc.c[k].y += C.la * x0.c[k].y + C.lb * nb.y;
  }
}

template <typename A>
__device__ __forceinline__ A norm2(const Spinor<A>& v) {
  A n = A(0);
#pragma unroll
  for (int k = 0; k < 12; k++) n = fma(v.c[k].x, v.c[k].x, fma(v.c[k].y, v.c[k].y, n));
  return n;
}

// One FP64 partial per (CTA, lane) of the thread-level values v (summed over the warps).
template <typename A, int NW>
__device__ __forceinline__ void write_partial(A v, A (*red)[32], double* dst, int w, int lane) {
  red[w][lane] = v;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < NW; k++) t += (double)red[k][lane];
    dst[lane] = t;
  }
}

// Sum over the slot's C partials of this lane's block (fixed order); valid in every thread.
__device__ __forceinline__ double slot_total(const double* part, int C, double* sc, int w,
                                             int lane) {
  if (w == 0) {
    double t = 0.0;
    for (int c = 0; c < C; c++) t += __ldcg(part + c * 32 + lane);
    sc[lane] = t;
  }
  __syncthreads();
  const double t = sc[lane];
  __syncthreads();
  return t;
}

// Launch variants (timed by the host's tuner): V = 0 two-slot ring, register budget for two
// CTAs per SM; V = 1 three-slot ring (two directions in flight); V = 2 two-slot ring, budget
// for three CTAs per SM.
__host__ __device__ constexpr int simd_rs(int v) { return v == 1 ? 3 : 2; }
__host__ __device__ constexpr int simd_minb(int p, int v) { return p == P64 ? 1 : v == 2 ? 3 : 2; }

template <int P, int LS, int V>
__global__ void __launch_bounds__(32 * LS / simd_nsl<P>(), simd_minb(P, V))
simd_local_kernel(const SimdArgs a) {
  constexpr int RS = simd_rs(V);
  using A = typename Prec<P>::acc;
  constexpr int NSL = simd_nsl<P>();
  constexpr int LSP = LS / NSL;    // warps; thread (lane, w) handles slices w + j LSP
  constexpr int NT = 32 * LSP;
  extern __shared__ __align__(128) unsigned char smem[];
  uint4* lraw0 = reinterpret_cast<uint4*>(smem);
  uint4* lraw1 = reinterpret_cast<uint4*>(smem + simd_lraw_bytes<P>());
  unsigned char* region = smem + 2 * simd_lraw_bytes<P>();
  uint4* ring = reinterpret_cast<uint4*>(region);   // during the hops
  A* buf = reinterpret_cast<A*>(region);            // afterwards
  __shared__ A red[LSP][32];
  __shared__ double sc[32];
  const int lane = threadIdx.x, w = threadIdx.y, tid = lane + 32 * w;
  const int C = a.C, slot = blockIdx.x % a.nslots, ci = blockIdx.x / a.nslots;
  if (slot >= a.nslots) return;
  unsigned* ctr = a.ctr + slot;
  double* part = a.partial + (long)slot * C * 32;
  unsigned nbar = 0;
  const Coef5<A> K = simd_coef<A>(a);
  const int NB = a.NB;
  const long sB = a.sB, sE = a.sE, sO = a.sO;
  const void* pin1 = a.trivial ? a.p : a.u;   // input of P1: D+ p (p itself when D+ = b)
  auto barrier = [&]() -> bool {
    ++nbar;
    return slot_barrier(ctr, nbar * (unsigned)C, a.wait_ns, a.err);
  };
  // One hop phase over the schedule `sch` (n entries) of output tables `tab`: the tile's links
  // and its table row are copied one tile ahead into the idle buffers, and the schedule entry
  // two tiles ahead is loaded while the current tile computes, so no global load sits between
  // a tile's start and its first neighbour copy.  `body(pos, row, live, lraw)` computes the
  // tile (row in shared memory).
  __shared__ __align__(16) uint32_t rows_s[2][8];
  auto phase = [&](const uint32_t* sch, int n, const uint32_t* tab, const void* links,
                   long lstride, long eg0, auto body) {
    auto prefetch = [&](uint4* lbuf, uint32_t* rbuf, uint32_t ent) {
      const int pos = (int)(ent & SIMD_POS_MASK);
      if (tid < 2) cp_async16<false>(rbuf + 4 * tid, tab + pos * 8 + 4 * tid);
      simd_prefetch_links<P>(lbuf, links, lstride, (long)pos * NB + eg0, ent >> 24, tid, NT);
    };
    uint32_t e_cur = ci < n ? __ldg(sch + ci) : 0u;
    uint32_t e_nxt = ci + C < n ? __ldg(sch + ci + C) : 0u;
    if (ci < n) prefetch(lraw0, rows_s[0], e_cur);
    int it = 0;
    for (int i = ci; i < n; i += C, it++) {
      const uint32_t e_nn = i + 2 * C < n ? __ldg(sch + i + 2 * C) : 0u;
      uint4* cur = (it & 1) ? lraw1 : lraw0;
      uint4* nxt = (it & 1) ? lraw0 : lraw1;
      cp_async_wait<0>();
      __syncthreads();   // every thread's copies of this tile (links, row) have landed
      if (i + C < n) prefetch(nxt, rows_s[(it + 1) & 1], e_nxt);
      body((int)(e_cur & SIMD_POS_MASK), rows_s[it & 1], e_cur >> 24, cur);
      e_cur = e_nxt;
      e_nxt = e_nn;
    }
    cp_async_wait<0>();
    __syncthreads();
  };

  for (int g = slot; g < a.ngroups; g += a.nslots) {
    const long eg0 = (long)g * 32;
    const long eg = eg0 + lane;   // this lane's block, as an element offset
    double rho, alpha = 0.0, beta = 0.0;
    // this lane's block takes part in this call (Schwarz colour)
    bool active = true;
    if (a.ncol > 1) {
      int bb = (int)(g * 32 + lane), bc[4];
#pragma unroll
      for (int m = 0; m < 4; m++) {
        bc[m] = bb % a.nbk[m];
        bb /= a.nbk[m];
      }
      const int colour = a.ncol == 2 ? (bc[0] + bc[1] + bc[2] + bc[3]) & 1
                                     : (bc[0] & 1) | (bc[1] & 1) << 1 | (bc[2] & 1) << 2 |
                                           (bc[3] & 1) << 3;
      active = (colour == a.col);
    }
    // ---- P0: r = f r_outer (gathered into the block layout), p = r, x = 0, u = D+ p
    {
      double f = a.num;
      if (a.den) f = sqrt(a.num / *a.den);
      A nrm = A(0);
      for (int pos = ci; pos < a.nBE; pos += C) {
        const long e = (long)pos * NB + eg;
        const int o = __ldg(a.fwd + e);
        Spinor<A> v[NSL];
#pragma unroll
        for (int j = 0; j < NSL; j++) {
          const int s = w + j * LSP;
          if (o < 0 || !active) {
            zero(v[j]);
          } else if (a.prec_outer == P64) {
            Spinor<double> q;
            load_spinor<P64>(q, a.r_outer, a.Vp_outer, o, s);
#pragma unroll
            for (int k = 0; k < 12; k++) v[j].c[k] = {A(q.c[k].x * f), A(q.c[k].y * f)};
          } else {
            Spinor<float> q;
            load_spinor<P32>(q, a.r_outer, a.Vp_outer, o, s);
            const A ff = A(f);
#pragma unroll
            for (int k = 0; k < 12; k++) v[j].c[k] = {A(q.c[k].x) * ff, A(q.c[k].y) * ff};
          }
          store_spinor<P>(a.r, sB, e, s, v[j]);
          store_spinor<P>(a.p, sB, e, s, v[j]);
          Spinor<A> zz;
          zero(zz);
          store_spinor<P>(a.x, sB, e, s, zz);
          round_to_storage<P>(v[j]);
          nrm += norm2(v[j]);
        }
        if (!a.trivial) {
          dplus_slices<A, LS, NSL, false>(v, buf, K, w, lane);
#pragma unroll
          for (int j = 0; j < NSL; j++) store_spinor<P>(a.u, sB, e, w + j * LSP, v[j]);
        }
      }
      write_partial<A, LSP>(nrm, red, part + ci * 32, w, lane);
      if (!barrier()) return;
      rho = slot_total(part, C, sc, w, lane);
    }
    for (int k = 0; k < a.l; k++) {
      const bool last = (k + 1 == a.l);
      // ---- P1: t = [D+ M5op^-1] Dh_oe (D+ p) on O
      phase(a.sch[0], a.nsch[0], a.nbrO, a.linksO, sO, eg0,
            [&](int pos, const uint32_t* row, uint32_t live, const uint4* lraw) {
              Spinor<A> acc[NSL];
              simd_hop_out<P, LS, false, RS>(acc, row, live, pin1, sB, NB, eg, w, lraw, ring, lane, tid);
              __syncthreads();   // the ring becomes the post buffer
#pragma unroll
              for (int j = 0; j < NSL; j++) to_buf(buf, acc[j], w + j * LSP, lane);
              __syncthreads();
              post_recurrence<A, LS, false>(buf, K, tid, NT);
              __syncthreads();
#pragma unroll
              for (int j = 0; j < NSL; j++) {
                from_buf(acc[j], buf, w + j * LSP, lane);
                store_spinor<P>(a.t, sO, (long)pos * NB + eg, w + j * LSP, acc[j]);
              }
            });
      if (!barrier()) return;
      // ---- P2: y = M5op p - 1/4 Dh_eo t on E; <p, A_s p> = ||y||^2 over the block
      {
        A nrm = A(0);
        const A hs = A(-0.25);
        phase(a.sch[1], a.nsch[1], a.nbrE, a.linksE, sE, eg0,
              [&](int pos, const uint32_t* row, uint32_t live, const uint4* lraw) {
                Spinor<A> acc[NSL];
                simd_hop_out<P, LS, false, RS>(acc, row, live, a.t, sO, NB, eg, w, lraw, ring, lane,
                                           tid);
                const long e = (long)pos * NB + eg;
#pragma unroll
                for (int j = 0; j < NSL; j++) {
                  const int s = w + j * LSP;
#pragma unroll
                  for (int q = 0; q < 12; q++) acc[j].c[q] = cscale(hs, acc[j].c[q]);
                  if (pos < a.nBE) add_m5<P, false>(acc[j], a.p, sB, e, s, LS, K);
                  nrm += norm2(acc[j]);
                  if (!last) store_spinor<P>(a.y, sE, e, s, acc[j]);
                }
              });
        write_partial<A, LSP>(nrm, red, part + ci * 32, w, lane);
        if (!barrier()) return;
        const double pap = slot_total(part, C, sc, w, lane);
        alpha = (pap > 0.0 && isfinite(pap)) ? rho / pap : 0.0;
      }
      if (last) {
        // ---- x += alpha p (the last iteration needs no new residual or direction)
        const A al = A(alpha);
        for (int pos = ci; pos < a.nBE; pos += C) {
          const long e = (long)pos * NB + eg;
#pragma unroll
          for (int j = 0; j < NSL; j++) {
            const int s = w + j * LSP;
            Spinor<A> xv, pv;
            ld_spinor<P>(xv, a.x, sB, e, s);
            ld_spinor<P>(pv, a.p, sB, e, s);
#pragma unroll
            for (int q = 0; q < 12; q++) {
              xv.c[q].x += al * pv.c[q].x;
              xv.c[q].y += al * pv.c[q].y;
            }
            store_spinor<P>(a.x, sB, e, s, xv);
          }
        }
        break;
      }
      // ---- P3: s = [M5op^-dag D+^dag] Dh_oe^dag y on O
      phase(a.sch[2], a.nsch[2], a.nbrO, a.linksO, sO, eg0,
            [&](int pos, const uint32_t* row, uint32_t live, const uint4* lraw) {
              Spinor<A> acc[NSL];
              simd_hop_out<P, LS, true, RS>(acc, row, live, a.y, sE, NB, eg, w, lraw, ring, lane, tid);
              __syncthreads();
#pragma unroll
              for (int j = 0; j < NSL; j++) to_buf(buf, acc[j], w + j * LSP, lane);
              __syncthreads();
              post_recurrence<A, LS, true>(buf, K, tid, NT);
              __syncthreads();
#pragma unroll
              for (int j = 0; j < NSL; j++) {
                from_buf(acc[j], buf, w + j * LSP, lane);
                store_spinor<P>(a.t, sO, (long)pos * NB + eg, w + j * LSP, acc[j]);
              }
            });
      if (!barrier()) return;
      // ---- P4: r -= alpha (M5op^dag y - 1/4 D+^dag Dh_eo^dag s) on BE; ||r||^2 -> beta
      {
        A nrm = A(0);
        const A al = A(alpha), hs = A(a.hs_b);
        phase(a.sch[3], a.nsch[3], a.nbrE, a.linksE, sE, eg0,
              [&](int pos, const uint32_t* row, uint32_t live, const uint4* lraw) {
                Spinor<A> acc[NSL];
                simd_hop_out<P, LS, true, RS>(acc, row, live, a.t, sO, NB, eg, w, lraw, ring, lane,
                                          tid);
                if (!a.trivial) {
                  __syncthreads();   // the ring becomes the slice-exchange buffer
                  dplus_slices<A, LS, NSL, true>(acc, buf, K, w, lane);
                }
                const long e = (long)pos * NB + eg;
#pragma unroll
                for (int j = 0; j < NSL; j++) {
                  const int s = w + j * LSP;
#pragma unroll
                  for (int q = 0; q < 12; q++) acc[j].c[q] = cscale(hs, acc[j].c[q]);
                  add_m5<P, true>(acc[j], a.y, sE, e, s, LS, K);
                  Spinor<A> rr;
                  ld_spinor<P>(rr, a.r, sB, e, s);
#pragma unroll
                  for (int q = 0; q < 12; q++) {
                    rr.c[q].x -= al * acc[j].c[q].x;
                    rr.c[q].y -= al * acc[j].c[q].y;
                  }
                  store_spinor<P>(a.r, sB, e, s, rr);
                  round_to_storage<P>(rr);
                  nrm += norm2(rr);
                }
              });
        write_partial<A, LSP>(nrm, red, part + ci * 32, w, lane);
        if (!barrier()) return;
        const double rr_new = slot_total(part, C, sc, w, lane);
        beta = (rho > 0.0 && isfinite(rr_new)) ? rr_new / rho : 0.0;
        rho = rr_new;
      }
      // ---- P5: x += alpha p, p = r + beta p, u = D+ p on BE
      {
        const A al = A(alpha), be = A(beta);
        for (int pos = ci; pos < a.nBE; pos += C) {
          const long e = (long)pos * NB + eg;
          Spinor<A> pv[NSL];
#pragma unroll
          for (int j = 0; j < NSL; j++) {
            const int s = w + j * LSP;
            Spinor<A> xv, rv;
            ld_spinor<P>(xv, a.x, sB, e, s);
            ld_spinor<P>(pv[j], a.p, sB, e, s);
            ld_spinor<P>(rv, a.r, sB, e, s);
#pragma unroll
            for (int q = 0; q < 12; q++) {
              xv.c[q].x += al * pv[j].c[q].x;
              xv.c[q].y += al * pv[j].c[q].y;
              pv[j].c[q].x = rv.c[q].x + be * pv[j].c[q].x;
              pv[j].c[q].y = rv.c[q].y + be * pv[j].c[q].y;
            }
            store_spinor<P>(a.x, sB, e, s, xv);
            store_spinor<P>(a.p, sB, e, s, pv[j]);
            round_to_storage<P>(pv[j]);
          }
          if (!a.trivial) {
            dplus_slices<A, LS, NSL, false>(pv, buf, K, w, lane);
#pragma unroll
            for (int j = 0; j < NSL; j++) store_spinor<P>(a.u, sB, e, w + j * LSP, pv[j]);
          }
        }
      }
      if (!barrier()) return;
    }
    // the slot's partial sums are reused by its next block group
    if (g + a.nslots < a.ngroups && !barrier()) return;
  }
}

}  // namespace dwf
