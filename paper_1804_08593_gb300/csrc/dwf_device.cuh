// Device-side building blocks: precision traits, complex arithmetic, site-major field
// access, and the spin projection of the Wilson hopping term.
//
// Field layout (one parity of a 5D field): [s][chunk][site], each chunk 16 bytes:
//   FP64: 12 chunks of one complex (double2), FP32: 6 chunks of two complex (float4),
//   FP16/BF16: 3 chunks of four complex (8 halves).
// Complex component k = spin*3 + colour.  A warp reads 32 consecutive sites of one chunk,
// i.e. 512 contiguous bytes, so every load and store is a full-width coalesced vector access.
//
// Link layout (one parity of output sites): [dir][chunk][site] with dir = 2*mu + back and
// 16-byte chunks holding the 9 complex elements k = a*3+b of U_mu(x) (forward hops) or
// U_mu(x-mu)^dag (backward hops) in order: FP64 9 chunks of one complex, FP32 5 chunks of
// two (the last half-empty), FP16/BF16 3 chunks of four (the last 3/4 empty).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwf {

enum PrecId { P64 = 0, P32 = 1, P16 = 2, PB16 = 3 };

template <int P> struct Prec;
template <> struct Prec<P64> {
  using acc = double;
  using link2 = double2;
  static constexpr int NCH = 12;   // 16-byte chunks per spinor
  static constexpr int NCHL = 9;   // 16-byte chunks per link
  static constexpr int BYTES = 8;  // bytes per real
};
template <> struct Prec<P32> {
  using acc = float;
  using link2 = float2;
  static constexpr int NCH = 6;
  static constexpr int NCHL = 5;
  static constexpr int BYTES = 4;
};
template <> struct Prec<P16> {
  using acc = float;
  using link2 = __half2;
  static constexpr int NCH = 3;
  static constexpr int NCHL = 3;
  static constexpr int BYTES = 2;
};
template <> struct Prec<PB16> {
  using acc = float;
  using link2 = __nv_bfloat162;
  static constexpr int NCH = 3;
  static constexpr int NCHL = 3;
  static constexpr int BYTES = 2;
};

template <typename A> struct cx {
  A x, y;
};

template <typename A> __device__ __forceinline__ cx<A> cmul(cx<A> a, cx<A> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * b accumulated into c
template <typename A> __device__ __forceinline__ void cfma(cx<A>& c, cx<A> a, cx<A> b) {
  c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
}
template <typename A> __device__ __forceinline__ cx<A> cadd(cx<A> a, cx<A> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename A> __device__ __forceinline__ cx<A> csub(cx<A> a, cx<A> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename A> __device__ __forceinline__ cx<A> mul_i(cx<A> a) { return {-a.y, a.x}; }
template <typename A> __device__ __forceinline__ cx<A> cscale(A s, cx<A> a) {
  return {s * a.x, s * a.y};
}

template <typename A> struct Spinor {
  cx<A> c[12];  // index spin*3 + colour
};

// ---------------------------------------------------------------------------------------
// Spinor load/store in the chunked site-major layout.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 h2f(uint32_t v, bool bf) {
  if (bf) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
    return __bfloat1622float2(h);
  }
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b, bool bf) {
  uint32_t r;
  if (bf) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    r = *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(a, b);
    r = *reinterpret_cast<uint32_t*>(&h);
  }
  return r;
}

// Read-only load of a field: through the non-coherent path (the field is not written during
// the kernel), or with COH through L2 only (a persistent kernel that reads, after a grid
// barrier, data other CTAs wrote earlier in the same launch).
template <bool COH, typename T>
__device__ __forceinline__ T ldf(const T* p) {
  if constexpr (COH) return __ldcg(p); else return __ldg(p);
}

template <int P, bool COH = false>
__device__ __forceinline__ void load_spinor(Spinor<typename Prec<P>::acc>& out, const void* base,
                                            long Vp, long site, int s) {
  constexpr int NCH = Prec<P>::NCH;
  const uint4* p = reinterpret_cast<const uint4*>(base) + ((long)s * NCH) * Vp + site;
  if constexpr (P == P64) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = ldf<COH>(reinterpret_cast<const double2*>(p + k * Vp));
      out.c[k] = {v.x, v.y};
    }
  } else if constexpr (P == P32) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = ldf<COH>(reinterpret_cast<const float4*>(p + k * Vp));
      out.c[2 * k] = {v.x, v.y};
      out.c[2 * k + 1] = {v.z, v.w};
    }
  } else {
    constexpr bool BF = (P == PB16);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v = ldf<COH>(p + k * Vp);
      float2 a = h2f(v.x, BF), b = h2f(v.y, BF), c = h2f(v.z, BF), d = h2f(v.w, BF);
      out.c[4 * k] = {a.x, a.y};
      out.c[4 * k + 1] = {b.x, b.y};
      out.c[4 * k + 2] = {c.x, c.y};
      out.c[4 * k + 3] = {d.x, d.y};
    }
  }
}

template <int P>
__device__ __forceinline__ void store_spinor(void* base, long Vp, long site, int s,
                                             const Spinor<typename Prec<P>::acc>& v) {
  constexpr int NCH = Prec<P>::NCH;
  uint4* p = reinterpret_cast<uint4*>(base) + ((long)s * NCH) * Vp + site;
  if constexpr (P == P64) {
#pragma unroll
    for (int k = 0; k < 12; k++)
      *reinterpret_cast<double2*>(p + k * Vp) = make_double2(v.c[k].x, v.c[k].y);
  } else if constexpr (P == P32) {
#pragma unroll
    for (int k = 0; k < 6; k++)
      *reinterpret_cast<float4*>(p + k * Vp) =
          make_float4(v.c[2 * k].x, v.c[2 * k].y, v.c[2 * k + 1].x, v.c[2 * k + 1].y);
  } else {
    constexpr bool BF = (P == PB16);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 w;
      w.x = f2h(v.c[4 * k].x, v.c[4 * k].y, BF);
      w.y = f2h(v.c[4 * k + 1].x, v.c[4 * k + 1].y, BF);
      w.z = f2h(v.c[4 * k + 2].x, v.c[4 * k + 2].y, BF);
      w.w = f2h(v.c[4 * k + 3].x, v.c[4 * k + 3].y, BF);
      p[k * Vp] = w;
    }
  }
}

// The 9 complex elements of one link (16-byte vector loads).
// read-only load: through the non-coherent path from global memory, or plain from shared
template <bool SMEM, typename T>
__device__ __forceinline__ T ldro(const T* p) {
  if constexpr (SMEM) return *p; else return __ldg(p);
}

// SMEM: base is the tile's links staged in shared memory ([dir][chunk][32 sites]).
template <int P, bool SMEM = false>
__device__ __forceinline__ void load_link9(cx<typename Prec<P>::acc> (&u)[9], const void* base,
                                           long Vp, long site, int dir) {
  constexpr int NCHL = Prec<P>::NCHL;
  const uint4* p = reinterpret_cast<const uint4*>(base) + (long)dir * NCHL * Vp + site;
  if constexpr (P == P64) {
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const double2 v = ldro<SMEM>(reinterpret_cast<const double2*>(p + k * Vp));
      u[k] = {v.x, v.y};
    }
  } else if constexpr (P == P32) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float4 v = ldro<SMEM>(reinterpret_cast<const float4*>(p + k * Vp));
      u[2 * k] = {v.x, v.y};
      u[2 * k + 1] = {v.z, v.w};
    }
    const float2 v = ldro<SMEM>(reinterpret_cast<const float2*>(p + 4 * Vp));
    u[8] = {v.x, v.y};
  } else {
    constexpr bool BF = (P == PB16);
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint4 v = ldro<SMEM>(p + k * Vp);
      float2 a = h2f(v.x, BF), b = h2f(v.y, BF), c = h2f(v.z, BF), d = h2f(v.w, BF);
      u[4 * k] = {a.x, a.y};
      u[4 * k + 1] = {b.x, b.y};
      u[4 * k + 2] = {c.x, c.y};
      u[4 * k + 3] = {d.x, d.y};
    }
    const float2 a = h2f(ldro<SMEM>(reinterpret_cast<const unsigned int*>(p + 2 * Vp)), BF);
    u[8] = {a.x, a.y};
  }
}

// Rounds a spinor to the values the storage precision would hold.
template <int P>
__device__ __forceinline__ void round_to_storage(Spinor<typename Prec<P>::acc>& v) {
  if constexpr (P == P16 || P == PB16) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const float2 f = h2f(f2h(v.c[k].x, v.c[k].y, P == PB16), P == PB16);
      v.c[k] = {f.x, f.y};
    }
  }
}

template <typename A> __device__ __forceinline__ void zero(Spinor<A>& s) {
#pragma unroll
  for (int k = 0; k < 12; k++) s.c[k] = {A(0), A(0)};
}

// ---------------------------------------------------------------------------------------
// One term of the Wilson hopping sum: acc += (1 + sgn*gamma_mu) U psi, using
// (1 + sgn*gamma_mu) = [[1, sgn*B], [sgn*B^dag, 1]] in the chiral basis, so the lower two
// spins are sgn * B^dag times the projected upper half-spinor h = psi_up + sgn*B psi_dn.
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.
// ---------------------------------------------------------------------------------------
// the projected upper half-spinor h = psi_up + sgn * B_mu psi_dn
template <typename A, int MU>
__device__ __forceinline__ void project_half(cx<A> (&h)[2][3], const Spinor<A>& psi, A sgn) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cx<A> p0 = psi.c[a], p1 = psi.c[3 + a], p2 = psi.c[6 + a], p3 = psi.c[9 + a];
    cx<A> b0, b1;  // B psi_dn
    if constexpr (MU == 0) {
      b0 = mul_i(p3); b0 = {-b0.x, -b0.y};
      b1 = mul_i(p2); b1 = {-b1.x, -b1.y};
    } else if constexpr (MU == 1) {
      b0 = {-p3.x, -p3.y};
      b1 = p2;
    } else if constexpr (MU == 2) {
      b0 = mul_i(p2); b0 = {-b0.x, -b0.y};
      b1 = mul_i(p3);
    } else {
      b0 = p2;
      b1 = p3;
    }
    h[0][a] = {p0.x + sgn * b0.x, p0.y + sgn * b0.y};
    h[1][a] = {p1.x + sgn * b1.x, p1.y + sgn * b1.y};
  }
}

// the same term with the link matrix u already in registers
template <int P, int MU>
__device__ __forceinline__ void hop_term_u(Spinor<typename Prec<P>::acc>& acc,
                                           const Spinor<typename Prec<P>::acc>& psi,
                                           const cx<typename Prec<P>::acc> (&u)[9],
                                           typename Prec<P>::acc sgn) {
  using A = typename Prec<P>::acc;
  cx<A> h[2][3];
  project_half<A, MU>(h, psi, sgn);
  cx<A> g[2][3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    g[0][a] = {A(0), A(0)};
    g[1][a] = {A(0), A(0)};
#pragma unroll
    for (int b = 0; b < 3; b++) {
      cfma(g[0][a], u[a * 3 + b], h[0][b]);
      cfma(g[1][a], u[a * 3 + b], h[1][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    acc.c[a] = cadd(acc.c[a], g[0][a]);
    acc.c[3 + a] = cadd(acc.c[3 + a], g[1][a]);
    cx<A> l0, l1;  // B^dag g
    if constexpr (MU == 0) {
      l0 = mul_i(g[1][a]);
      l1 = mul_i(g[0][a]);
    } else if constexpr (MU == 1) {
      l0 = g[1][a];
      l1 = {-g[0][a].x, -g[0][a].y};
    } else if constexpr (MU == 2) {
      l0 = mul_i(g[0][a]);
      l1 = mul_i(g[1][a]); l1 = {-l1.x, -l1.y};
    } else {
      l0 = g[0][a];
      l1 = g[1][a];
    }
    acc.c[6 + a] = {acc.c[6 + a].x + sgn * l0.x, acc.c[6 + a].y + sgn * l0.y};
    acc.c[9 + a] = {acc.c[9 + a].x + sgn * l1.x, acc.c[9 + a].y + sgn * l1.y};
  }
}

template <int P, int MU, bool SMEM = false>
__device__ __forceinline__ void hop_term(Spinor<typename Prec<P>::acc>& acc,
                                         const Spinor<typename Prec<P>::acc>& psi,
                                         const void* links, long Vp, long site, int dir,
                                         typename Prec<P>::acc sgn) {
  cx<typename Prec<P>::acc> u[9];
  load_link9<P, SMEM>(u, links, Vp, site, dir);
  hop_term_u<P, MU>(acc, psi, u, sgn);
}

// Neighbour table entries: index of the neighbour in the other parity's site order; bit 31
// marks a hop that crosses a block face (skipped by the block-local operator); bit 30 marks a
// neighbour that lives in the block's own halo array (exact block operator).
constexpr uint32_t NBR_FACE = 0x80000000u;
constexpr uint32_t NBR_HALO = 0x40000000u;
constexpr uint32_t NBR_IDX = 0x3fffffffu;

// ---------------------------------------------------------------------------------------
// Deterministic grid reduction: per-CTA partials, the last CTA of each segment sums its
// segment's partials in a fixed order and applies a finalize operation.
// ---------------------------------------------------------------------------------------
enum FinOp {
  FIN_STORE = 0,   // res[seg] = v
  FIN_ALPHA = 1,   // alpha[seg] = rho[seg] / v   (v = <p, A p>)
  FIN_BETA = 2,    // beta[seg] = v / rho[seg]; rho[seg] = v; conv if v <= stop2
  FIN_NONE = 3,
  FIN_ALPHA2 = 4   // alpha[seg] = rho[seg] / (v + extra[seg])
};

struct RedArgs {
  double* partial;      // [gridDim.x * NV]
  unsigned* counter;    // [nseg], zero between uses
  int cps;              // CTAs per segment
  int op;               // FinOp
  double* res;          // [nseg * NV]
  double* rho;          // [nseg]
  double* alpha;        // [nseg]
  double* beta;         // [nseg]
  const double* stop2;  // per-segment stop threshold on v, nullable
  int* conv;            // conv[seg] set to 1 when v <= stop2[seg], nullable
  const double* extra;  // FIN_ALPHA2: partial sum from a previous launch
  double* hist;         // FIN_BETA: hist[*hist_idx] = v; FIN_ALPHA: the curvature (nullable)
  const int* hist_idx;
  int hist_cap;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values per thread; result valid in thread 0.  scratch: >= 32*NV values.
// FP32 kernels sum their CTA in FP32 (GB300's FP64 pipe is narrow) and hand one FP64 partial
// per CTA to the grid-level sum.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* scratch) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
  for (int i = 0; i < NV; i++) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; i++) scratch[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) {
      T t = lane < nw ? scratch[lane * NV + i] : T(0);
      v[i] = warp_sum(t);
    }
  }
}

template <int NV>
__device__ void finalize_value(const RedArgs& r, int seg, const double (&v)[NV]) {
#pragma unroll
  for (int i = 0; i < NV; i++)
    if (r.res) r.res[seg * NV + i] = v[i];
  const double x = v[0];
  if (r.op == FIN_ALPHA || r.op == FIN_ALPHA2) {
    const double rho = r.rho[seg];
    const double pap = r.op == FIN_ALPHA2 ? x + r.extra[seg] : x;
    r.alpha[seg] = (pap > 0.0 && isfinite(pap)) ? rho / pap : 0.0;
    if (r.hist && *r.hist_idx < r.hist_cap) r.hist[*r.hist_idx] = pap;
  } else if (r.op == FIN_BETA) {
    const double rho = r.rho[seg];
    r.beta[seg] = (rho > 0.0 && isfinite(x)) ? x / rho : 0.0;
    r.rho[seg] = x;
    if (r.stop2 && r.conv && (x <= r.stop2[seg] || !isfinite(x))) r.conv[seg] = 1;
    if (r.hist && *r.hist_idx < r.hist_cap) r.hist[*r.hist_idx] = x;
  }
}

// Called by every thread of the CTA after its per-thread values are known, for the 32-site
// tile `tile` of segment `seg` whose tiles are [first, first + ntiles).  The last tile of the
// segment to arrive sums the segment's partials in a fixed order (deterministic) and
// finalizes.  Returns normally in every thread (usable inside a persistent tile loop).
template <int NV, typename T>
__device__ void grid_reduce_seg(const RedArgs& r, T (&v)[NV], double* scratch, long tile,
                                int seg, long first, int ntiles) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  block_sum<NV, T>(v, reinterpret_cast<T*>(scratch));
  __shared__ unsigned is_last;
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) r.partial[tile * NV + i] = (double)v[i];
    __threadfence();
    const unsigned prev = atomicAdd(&r.counter[seg], 1u);
    is_last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double s[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) s[i] = 0.0;
    for (int k = tid; k < ntiles; k += nthr)
#pragma unroll
      for (int i = 0; i < NV; i++) s[i] += __ldcg(&r.partial[(first + k) * NV + i]);
    block_sum<NV, double>(s, scratch);
    if (tid == 0) {
      finalize_value<NV>(r, seg, s);
      r.counter[seg] = 0u;
    }
  }
  __syncthreads();
}

// Uniform segments of r.cps tiles (tile = blockIdx.x).
template <int NV, typename T>
__device__ void grid_reduce(const RedArgs& r, T (&v)[NV], double* scratch) {
  const int seg = blockIdx.x / r.cps;
  grid_reduce_seg<NV, T>(r, v, scratch, blockIdx.x, seg, (long)seg * r.cps, r.cps);
}

// Per-problem description of a batched (concatenated) site space: problem = segment.
// Fifth-dimension coefficients of a stage in one arithmetic type, computed on the host so
// that FP32 kernels run no FP64 instructions (GB300's FP64 pipe is narrow):
// M5op = la + lb K with walls -mf, D+ = db + dc K, and for the recurrence post r = lb/la,
// inva = 1/la, kappa = r mf / (1 + mf (-r)^Ls), pre = extra factor of D+ M5op^-1.
template <typename A>
struct Coef5 {
  A la, lb, mf, db, dc, r, inva, kappa, pre;
};
template <typename A>
inline Coef5<A> make_coef5(double la, double lb, double mf, double db, double dc, double pre,
                           int Ls) {
  const double r = la != 0.0 ? lb / la : 0.0;
  double pw = 1.0;
  for (int i = 0; i < Ls; i++) pw *= -r;
  const double kappa = r * mf / (1.0 + mf * pw);
  return {A(la), A(lb), A(mf), A(db), A(dc), A(r), A(la != 0.0 ? 1.0 / la : 0.0), A(kappa),
          A(pre)};
}

struct BatchSeg {
  const void* mat[3];   // D+ M5op^-1, M5op^-dag D+^dag, D+^dag in the accumulation type
  double l_alpha, l_beta, mf, db, dc;
  Coef5<double> k64;    // the same coefficients for the stage kernels (pre = 1)
  Coef5<float> k32;
  int Vh;               // sites of one parity of this problem
  int first_tile;       // first 32-site tile of the problem in the concatenation
  int ntiles;
};

// Writes the 9 complex elements v[k] = (re, im) of one link as 16-byte chunks.
template <int P>
__device__ __forceinline__ void store_link9(void* out, long Vp, long idx, int d,
                                            const double (&re)[9], const double (&im)[9]) {
  constexpr int NCHL = Prec<P>::NCHL;
  uint4* o = reinterpret_cast<uint4*>(out) + (long)d * NCHL * Vp + idx;
  if constexpr (P == P64) {
    for (int k = 0; k < 9; k++) *reinterpret_cast<double2*>(o + k * Vp) = make_double2(re[k], im[k]);
  } else if constexpr (P == P32) {
    for (int k = 0; k < 5; k++) {
      const int a = 2 * k, b = 2 * k + 1;
      *reinterpret_cast<float4*>(o + k * Vp) =
          make_float4((float)re[a], (float)im[a], b < 9 ? (float)re[b] : 0.f,
                      b < 9 ? (float)im[b] : 0.f);
    }
  } else {
    constexpr bool BF = (P == PB16);
    for (int k = 0; k < 3; k++) {
      uint32_t w[4];
      for (int j = 0; j < 4; j++) {
        const int e = 4 * k + j;
        w[j] = e < 9 ? f2h((float)re[e], (float)im[e], BF) : 0u;
      }
      o[k * Vp] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

}  // namespace dwf
