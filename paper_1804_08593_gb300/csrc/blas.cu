// Vector kernels of the Krylov solvers: the fused CG update (x += alpha p, p = r + beta p,
// u = D+ p), precision casts with a scale and a fused dot product, and small vector ops.
// All use CTA = 32 sites x Ls slices so that reductions are segmented per lattice block
// exactly like the operator stages (segment = CTA index / (Vhb_pad / 32)).
#include <atomic>
#include <type_traits>

#include "dwf_internal.h"
#include "vec_tile.cuh"

namespace dwf {

// Sets a kernel's dynamic shared memory limit once per device (one bit per device ordinal).
template <typename K>
static cudaError_t set_smem_once(K kernel, std::atomic<uint64_t>& done, int bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
  if (done.load() & bit) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <int P, int LS>
__global__ void __launch_bounds__(32 * LS) vec_kernel(const VecArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  vec_tile<P, LS>(a, blockIdx.x, gridDim.x, smem_raw);
}

template <int P, int LS>
static cudaError_t vec_launch(const VecArgs& a, cudaStream_t st) {
  using A = typename Prec<P>::acc;
  const size_t sm = a.do_u ? (size_t)LS * 24 * 32 * sizeof(A) : 0;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e = set_smem_once(vec_kernel<P, LS>, attr, (int)(LS * 24 * 32 * sizeof(A)));
  if (e != cudaSuccess) return e;
  vec_kernel<P, LS><<<dim3((unsigned)(a.Vp / 32)), dim3(32, LS), sm, st>>>(a);
  return cudaGetLastError();
}

template <int P>
static cudaError_t vec_dispatch(const VecArgs& a, int Ls, cudaStream_t st) {
  switch (Ls) {
    case 4: return vec_launch<P, 4>(a, st);
    case 6: return vec_launch<P, 6>(a, st);
    case 8: return vec_launch<P, 8>(a, st);
    case 10: return vec_launch<P, 10>(a, st);
    case 12: return vec_launch<P, 12>(a, st);
    case 16: return vec_launch<P, 16>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vec(int prec, const VecArgs& a, int Ls, cudaStream_t st) {
  switch (prec) {
    case P64: return vec_dispatch<P64>(a, Ls, st);
    case P32: return vec_dispatch<P32>(a, Ls, st);
    case P16: return vec_dispatch<P16>(a, Ls, st);
    default: return vec_dispatch<PB16>(a, Ls, st);
  }
}

// ---------------------------------------------------------------------------------------
// Casts between precisions: out = in * f, f = sqrt(num / *den) (or num), optionally 1/f;
// optional reduction <dotv, out> over what was stored.
// ---------------------------------------------------------------------------------------
template <int PI, int PO>
__global__ void cast_kernel(const CastArgs a) {
  using AI = typename Prec<PI>::acc;
  using AO = typename Prec<PO>::acc;
  __shared__ double scratch[32];
  int seg = 0;
  if (a.tile_seg) {
    seg = a.tile_seg[blockIdx.x];
    if (a.stop && a.stop[seg]) return;
  } else if (a.stop && *a.stop) {
    return;
  }
  const int lane = threadIdx.x, s = threadIdx.y;
  const long site = (long)blockIdx.x * 32 + lane;
  // the scale factor is computed once per CTA (FP64 is slow on this part) and applied in
  // the wider of the two accumulation types
  using AW = typename std::conditional<(PI == P64 || PO == P64), double, float>::type;
  __shared__ double fsh;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double f = a.num;
    if (a.den) {
      const double d = *a.den;
      f = (d > 0.0 && isfinite(d)) ? sqrt(a.num / d) : 1.0;
    }
    fsh = a.invert ? 1.0 / f : f;
  }
  __syncthreads();
  const AW f = AW(fsh);
  Spinor<AI> v;
  if (a.in_map) {   // a gather from another site order
    const int j = a.in_map[site];
    if (j >= 0)
      load_spinor<PI>(v, a.in, a.Vp_in, j, s);
    else
      zero(v);
  } else {
    load_spinor<PI>(v, a.in, a.Vp, site, s);
  }
  Spinor<AO> w;
#pragma unroll
  for (int k = 0; k < 12; k++) w.c[k] = {AO((AW)v.c[k].x * f), AO((AW)v.c[k].y * f)};
  if (a.out) store_spinor<PO>(a.out, a.Vp, site, s, w);   // no out: the reduction only
  if (a.out2) store_spinor<PO>(a.out2, a.Vp, site, s, w);
  round_to_storage<PO>(w);   // from here on: the values as stored
  if (a.out3) {
    // u_s = db w_s + dc (P- w_{s+1} + P+ w_{s-1}),  w_{Ls} = -mf w_0, w_{-1} = -mf w_{Ls-1}:
    // the slices of the site are the CTA's other warps, exchanged through shared memory
    extern __shared__ __align__(128) unsigned char cast_smem[];
    AO* buf = reinterpret_cast<AO*>(cast_smem);
    const int Ls = blockDim.y;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      buf[(s * 24 + 2 * k) * 32 + lane] = w.c[k].x;
      buf[(s * 24 + 2 * k + 1) * 32 + lane] = w.c[k].y;
    }
    __syncthreads();
    AO db, dc, mf;
    if constexpr (sizeof(AO) == 8) {
      db = a.db; dc = a.dc; mf = a.mf;
    } else {
      db = a.dbf; dc = a.dcf; mf = a.mff;
    }
    const int su = s + 1 < Ls ? s + 1 : 0, sd = s > 0 ? s - 1 : Ls - 1;
    const AO fu = (s + 1 < Ls) ? AO(1) : -mf, fd = (s > 0) ? AO(1) : -mf;
    Spinor<AO> u;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const int sn = k < 6 ? sd : su;
      const AO f = k < 6 ? fd : fu;
      u.c[k].x = db * w.c[k].x + dc * f * buf[(sn * 24 + 2 * k) * 32 + lane];
      u.c[k].y = db * w.c[k].y + dc * f * buf[(sn * 24 + 2 * k + 1) * 32 + lane];
    }
    store_spinor<PO>(a.out3, a.Vp, site, s, u);
  }
  if (a.red.partial) {
    AO part = AO(0);
    if (a.dotv) {
      Spinor<AO> d;
      load_spinor<PO>(d, a.dotv, a.Vp, site, s);
#pragma unroll
      for (int k = 0; k < 12; k++) part = fma(d.c[k].x, w.c[k].x, fma(d.c[k].y, w.c[k].y, part));
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) part = fma(w.c[k].x, w.c[k].x, fma(w.c[k].y, w.c[k].y, part));
    }
    AO vv[1] = {part};
    if (a.tile_seg)
      grid_reduce_seg<1, AO>(a.red, vv, scratch, blockIdx.x, seg, a.segp[seg].first_tile,
                             a.segp[seg].ntiles);
    else
      grid_reduce<1, AO>(a.red, vv, scratch);
  }
}

template <int PI, int PO>
static cudaError_t cast_go(const CastArgs& a, dim3 g, dim3 b, cudaStream_t st) {
  using AO = typename Prec<PO>::acc;
  static std::atomic<uint64_t> attr{0};   // room for the D+ exchange of the largest Ls
  cudaError_t e = set_smem_once(cast_kernel<PI, PO>, attr, (int)(16 * 24 * 32 * sizeof(AO)));
  if (e != cudaSuccess) return e;
  const size_t sm = a.out3 ? (size_t)b.y * 24 * 32 * sizeof(AO) : 0;
  cast_kernel<PI, PO><<<g, b, sm, st>>>(a);
  return cudaGetLastError();
}

template <int PI>
static cudaError_t cast_out(int pout, const CastArgs& a, dim3 g, dim3 b, cudaStream_t st) {
  switch (pout) {
    case P64: return cast_go<PI, P64>(a, g, b, st);
    case P32: return cast_go<PI, P32>(a, g, b, st);
    case P16: return cast_go<PI, P16>(a, g, b, st);
    default: return cast_go<PI, PB16>(a, g, b, st);
  }
}

cudaError_t launch_cast(int pin, int pout, const CastArgs& a, int Ls, cudaStream_t st) {
  dim3 g((unsigned)(a.Vp / 32)), b(32, Ls);
  switch (pin) {
    case P64: return cast_out<P64>(pout, a, g, b, st);
    case P32: return cast_out<P32>(pout, a, g, b, st);
    case P16: return cast_out<P16>(pout, a, g, b, st);
    default: return cast_out<PB16>(pout, a, g, b, st);
  }
}

// ---------------------------------------------------------------------------------------
// Small vector ops.
// ---------------------------------------------------------------------------------------
template <int P, int PX>
__global__ void vop_kernel(const VopArgs a) {
  using A = typename Prec<P>::acc;
  using AX = typename Prec<PX>::acc;
  __shared__ double scratch[32];
  int seg = 0;
  if (a.tile_seg) {
    seg = a.tile_seg[blockIdx.x];
    if (a.stop && a.stop[seg]) return;
  } else if (a.stop && *a.stop) {
    return;
  }
  const int lane = threadIdx.x, s = threadIdx.y;
  const long site = (long)blockIdx.x * 32 + lane;
  double acc = 0.0;
  Spinor<A> y;
  switch (a.op) {
    case VOP_ZERO:
      zero(y);
      store_spinor<P>(a.y, a.Vp, site, s, y);
      break;
    case VOP_COPY:
      load_spinor<P>(y, a.x, a.Vp, site, s);
      store_spinor<P>(a.y, a.Vp, site, s, y);
      break;
    case VOP_AXPY: {
      const double c = a.sa * (a.ap ? *a.ap : 1.0);
      Spinor<A> x;
      load_spinor<P>(x, a.x, a.Vp, site, s);
      load_spinor<P>(y, a.y, a.Vp, site, s);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        y.c[k].x += A(c) * x.c[k].x;
        y.c[k].y += A(c) * x.c[k].y;
      }
      store_spinor<P>(a.y, a.Vp, site, s, y);
      break;
    }
    case VOP_XMY_NORM: {
      Spinor<A> x;
      load_spinor<P>(x, a.x, a.Vp, site, s);
      load_spinor<P>(y, a.y, a.Vp, site, s);
      A part = A(0);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        y.c[k].x = x.c[k].x - y.c[k].x;
        y.c[k].y = x.c[k].y - y.c[k].y;
        part = fma(y.c[k].x, y.c[k].x, fma(y.c[k].y, y.c[k].y, part));
      }
      acc = (double)part;
      store_spinor<P>(a.y, a.Vp, site, s, y);
      break;
    }
    case VOP_NORM: {
      load_spinor<P>(y, a.x, a.Vp, site, s);
      A part = A(0);
#pragma unroll
      for (int k = 0; k < 12; k++) part = fma(y.c[k].x, y.c[k].x, fma(y.c[k].y, y.c[k].y, part));
      acc = (double)part;
      break;
    }
    case VOP_DOT: {
      Spinor<A> x;
      load_spinor<P>(x, a.x, a.Vp, site, s);
      load_spinor<P>(y, a.y, a.Vp, site, s);
      A part = A(0);
#pragma unroll
      for (int k = 0; k < 12; k++) part = fma(x.c[k].x, y.c[k].x, fma(x.c[k].y, y.c[k].y, part));
      acc = (double)part;
      break;
    }
    case VOP_ADD_CAST: {
      Spinor<AX> x;
      load_spinor<PX>(x, a.x, a.Vp, site, s);
      load_spinor<P>(y, a.y, a.Vp, site, s);
      const double c = a.sa * (a.ap ? *a.ap : 1.0);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        y.c[k].x += A(c * (double)x.c[k].x);
        y.c[k].y += A(c * (double)x.c[k].y);
      }
      store_spinor<P>(a.y, a.Vp, site, s, y);
      break;
    }
  }
  if (a.red.partial) {
    double vv[1] = {acc};
    if (a.tile_seg)
      grid_reduce_seg<1, double>(a.red, vv, scratch, blockIdx.x, seg, a.segp[seg].first_tile,
                                 a.segp[seg].ntiles);
    else
      grid_reduce<1, double>(a.red, vv, scratch);
  }
}

template <int P>
static cudaError_t vop_px(int px, const VopArgs& a, dim3 g, dim3 b, cudaStream_t st) {
  switch (px) {
    case P64: vop_kernel<P, P64><<<g, b, 0, st>>>(a); break;
    case P32: vop_kernel<P, P32><<<g, b, 0, st>>>(a); break;
    case P16: vop_kernel<P, P16><<<g, b, 0, st>>>(a); break;
    default: vop_kernel<P, PB16><<<g, b, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_vop(int prec, int prec_x, const VopArgs& a, int Ls, cudaStream_t st) {
  dim3 g((unsigned)(a.Vp / 32)), b(32, Ls);
  if (a.op != VOP_ADD_CAST) prec_x = prec;
  switch (prec) {
    case P64: return vop_px<P64>(prec_x, a, g, b, st);
    case P32: return vop_px<P32>(prec_x, a, g, b, st);
    case P16: return vop_px<P16>(prec_x, a, g, b, st);
    default: return vop_px<PB16>(prec_x, a, g, b, st);
  }
}

}  // namespace dwf
