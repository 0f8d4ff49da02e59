// The fused CG update (x += alpha p, p = r + beta p, u = D+ p) of one 32-site tile, shared by
// the update kernel and by persistent kernels that run it as one of their phases.
#pragma once

#include <type_traits>

#include "dwf_internal.h"

namespace dwf {

// Completion counting without data: returns true in every thread of the last CTA to finish
// (of `total` CTAs that count on this counter).
__device__ __forceinline__ bool last_cta(unsigned* counter, unsigned total) {
  __shared__ unsigned is_last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == total - 1u);
  }
  __syncthreads();
  return is_last != 0u;
}

// z = f * src[j] converted to the accumulation type of P (the product in the wider type)
template <int PZ, int P>
__device__ __forceinline__ void load_z_as(Spinor<typename Prec<P>::acc>& r, const VecArgs& a,
                                          long j, int s, double f) {
  using A = typename Prec<P>::acc;
  using AZ = typename Prec<PZ>::acc;
  using AW = typename std::conditional<(PZ == P64 || P == P64), double, float>::type;
  Spinor<AZ> v;
  load_spinor<PZ>(v, a.z_src, a.z_vp, j, s);
  const AW fw = AW(f);
#pragma unroll
  for (int k = 0; k < 12; k++) r.c[k] = {A((AW)v.c[k].x * fw), A((AW)v.c[k].y * fw)};
}

// The CG update of one 32-site tile (all Ls slices; thread (lane, s)); ntiles_all: the CTAs that
// count on the single-segment completion counter.  COH: inputs written earlier in the same
// launch (persistent kernels) are read through L2.
template <int P, int LS, bool COH = false>
__device__ __forceinline__ void vec_tile(const VecArgs& a, long tile, unsigned ntiles_all,
                                         unsigned char* smem_raw) {
  using A = typename Prec<P>::acc;
  const int lane = threadIdx.x, s = threadIdx.y;
  const long site = tile * 32 + lane;
  int seg;
  double dbv = a.db, dcv = a.dc, mfv = a.mf;
  if (a.tile_seg) {
    seg = a.tile_seg[tile];
    if (a.stop && a.stop[seg]) return;
    dbv = a.segp[seg].db;
    dcv = a.segp[seg].dc;
    mfv = a.segp[seg].mf;
  } else {
    if (a.stop && *a.stop) return;
    seg = (int)(tile / a.seg_cps);
  }

  Spinor<A> p;
  load_spinor<P, COH>(p, a.p, a.Vp, site, s);
  if (a.do_x) {
    const A al = A(a.alpha[seg]);
    Spinor<A> x;
    load_spinor<P, COH>(x, a.x, a.Vp, site, s);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x.c[k].x += al * p.c[k].x;
      x.c[k].y += al * p.c[k].y;
    }
    store_spinor<P>(a.x, a.Vp, site, s, x);
  }
  if (a.do_p) {
    const A be = A(a.beta[seg]);
    Spinor<A> r;
    if (a.z_src) {
      // the scale once per CTA (FP64 is slow on this part)
      __shared__ double zf;
      if (threadIdx.x == 0 && threadIdx.y == 0) {
        double f = a.z_num;
        if (a.z_den) {
          const double d = *a.z_den;
          f = (d > 0.0 && isfinite(d)) ? sqrt(a.z_num / d) : 1.0;
        }
        zf = 1.0 / f;
      }
      __syncthreads();
      const long j = a.z_map ? (long)a.z_map[site] : site;
      if (j < 0) {
        zero(r);
      } else {
        switch (a.z_prec) {
          case P64: load_z_as<P64, P>(r, a, j, s, zf); break;
          case P32: load_z_as<P32, P>(r, a, j, s, zf); break;
          case P16: load_z_as<P16, P>(r, a, j, s, zf); break;
          default: load_z_as<PB16, P>(r, a, j, s, zf);
        }
      }
    } else {
      load_spinor<P, COH>(r, a.r, a.Vp, site, s);
    }
#pragma unroll
    for (int k = 0; k < 12; k++) {
      p.c[k].x = r.c[k].x + be * p.c[k].x;
      p.c[k].y = r.c[k].y + be * p.c[k].y;
    }
    store_spinor<P>(a.p, a.Vp, site, s, p);
    round_to_storage<P>(p);
  }
  if (a.do_u) {
    // u_s = db p_s + dc (P- p_{s+1} + P+ p_{s-1}),  p_{Ls} = -mf p_0, p_{-1} = -mf p_{Ls-1}
    A* buf = reinterpret_cast<A*>(smem_raw);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      buf[(s * 24 + 2 * k) * 32 + lane] = p.c[k].x;
      buf[(s * 24 + 2 * k + 1) * 32 + lane] = p.c[k].y;
    }
    __syncthreads();
    const int su = s + 1 < LS ? s + 1 : 0, sd = s > 0 ? s - 1 : LS - 1;
    const A fu = (s + 1 < LS) ? A(1) : A(-mfv), fd = (s > 0) ? A(1) : A(-mfv);
    const A db = A(dbv), dc = A(dcv);
    Spinor<A> u;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const int sn = k < 6 ? sd : su;
      const A f = k < 6 ? fd : fu;
      u.c[k].x = db * p.c[k].x + dc * f * buf[(sn * 24 + 2 * k) * 32 + lane];
      u.c[k].y = db * p.c[k].y + dc * f * buf[(sn * 24 + 2 * k + 1) * 32 + lane];
    }
    store_spinor<P>(a.u, a.Vp, site, s, u);
  }
  if (a.red.counter) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (a.tile_seg) {
      // per problem: the last tile of the problem copies its convergence flag to its stop
      // flag and counts the iteration
      if (last_cta(a.red.counter + seg, a.segp[seg].ntiles) && tid == 0) {
        if (a.stop_out && a.conv_in && a.conv_in[seg]) a.stop_out[seg] = 1;
        if (a.iter) a.iter[seg] += 1;
        a.red.counter[seg] = 0u;
      }
    } else if (last_cta(a.red.counter, ntiles_all)) {
      if (tid == 0) {
        if (a.stop_out && a.conv_in && *a.conv_in) *a.stop_out = 1;
        if (a.iter) *a.iter += 1;
        a.red.counter[0] = 0u;
      }
    }
  }
}

}  // namespace dwf
