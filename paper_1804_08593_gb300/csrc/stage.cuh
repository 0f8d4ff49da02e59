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
// CTA = 32 consecutive sites x all Ls slices (thread (lane, s)).  Links are read once per site
// by the first warp and served from L1 to the other Ls-1 warps; the Ls x Ls post matrix is a
// shared-memory column GEMM over the CTA's 32 sites x 24 reals.  The epilogue optionally
// fuses the CG residual update r -= alpha * out and a deterministic ||.||^2 reduction.
#pragma once

#include "dwf_device.cuh"

namespace dwf {

enum LocalMode { LOC_NONE = 0, LOC_M5 = 1, LOC_M5DAG = 2 };
enum EpiMode { EPI_STORE = 0, EPI_NORM = 1, EPI_CG_R = 2 };

struct StageArgs {
  const void* in;        // hop input, parity 1-p
  const void* in_halo;   // hop input for NBR_HALO neighbours (exact block operator)
  long Vp_in, Vp_halo;   // site strides of in / in_halo
  const int* link_site;  // nullable: links of output site i are at link_site[i]
  long Vp_link;          // site stride of the link array
  int skip_halo;         // treat NBR_HALO neighbours as absent
  void* out;             // output, parity p (EPI_STORE / EPI_NORM)
  const void* in2;       // local-term input, parity p (nullable if LOC_NONE)
  void* r;               // EPI_CG_R: residual updated in place
  const void* links;     // links of parity p: [8][9][Vp]
  const uint32_t* nbr;   // neighbours of parity p: [8][Vp]
  const void* post;      // [2][Ls][Ls] in the accumulation type, nullable
  long Vp;               // site stride of out / in2 / r and of the neighbour table
  int Vhb, Vhb_pad;
  double hop_scale;
  int local_mode;
  double l_alpha, l_beta, mf;
  int epi;
  const double* alpha;   // EPI_CG_R: per-segment alpha
  int seg_cps;           // CTAs per scalar/reduction segment (Vp/32: one global segment)
  const int* stop;       // nullable: skip everything when *stop != 0
  RedArgs red;
};

template <int P, int D, bool DAG, bool BLOCKED>
__device__ __forceinline__ void hop_dir(Spinor<typename Prec<P>::acc>& acc, const StageArgs& a,
                                        long site, long lsite, int s) {
  using A = typename Prec<P>::acc;
  const uint32_t nb = __ldg(a.nbr + (long)D * a.Vp + site);
  Spinor<A> psi;
  if constexpr (BLOCKED) {
    if (nb & NBR_FACE) return;
    if (nb & NBR_HALO) {
      if (a.skip_halo) return;
      load_spinor<P>(psi, a.in_halo, a.Vp_halo, (long)(nb & NBR_IDX), s);
    } else {
      load_spinor<P>(psi, a.in, a.Vp_in, (long)(nb & NBR_IDX), s);
    }
  } else {
    load_spinor<P>(psi, a.in, a.Vp_in, (long)(nb & NBR_IDX), s);
  }
  // forward hop: (1 - gamma_mu), backward: (1 + gamma_mu); the adjoint swaps them.
  constexpr bool back = (D & 1) != 0;
  const A sgn = (back != DAG) ? A(1) : A(-1);
  hop_term<P, D / 2>(acc, psi, a.links, a.Vp_link, lsite, D, sgn);
}

template <int P, int LS, bool DAG, bool BLOCKED>
__global__ void __launch_bounds__(32 * LS) stage_kernel(const StageArgs a) {
  using A = typename Prec<P>::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_scratch[32];
  if (a.stop && *a.stop) return;

  const int lane = threadIdx.x, s = threadIdx.y;
  const int tid = lane + 32 * s;
  constexpr int NT = 32 * LS;
  const long site = (long)blockIdx.x * 32 + lane;
  const int cps = a.Vhb_pad >> 5;
  const int jl = (blockIdx.x % cps) * 32 + lane;
  const bool valid = jl < a.Vhb;

  Spinor<A> acc;
  zero(acc);
  if (valid) {
    const long lsite = a.link_site ? (long)__ldg(a.link_site + site) : site;
    hop_dir<P, 0, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 1, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 2, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 3, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 4, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 5, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 6, DAG, BLOCKED>(acc, a, site, lsite, s);
    hop_dir<P, 7, DAG, BLOCKED>(acc, a, site, lsite, s);
  }

  if (a.post != nullptr) {
    // Dense per-chirality Ls x Ls matrix along s: buf[s][24][32] holds the CTA's hop results;
    // each thread owns whole (component, site) columns and writes them back in place.
    A* buf = reinterpret_cast<A*>(smem_raw);
    A* mat = buf + LS * 24 * 32;
    const A* pm = reinterpret_cast<const A*>(a.post);
    for (int i = tid; i < 2 * LS * LS; i += NT) mat[i] = pm[i];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      buf[(s * 24 + 2 * k) * 32 + lane] = acc.c[k].x;
      buf[(s * 24 + 2 * k + 1) * 32 + lane] = acc.c[k].y;
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
    for (int k = 0; k < 12; k++) {
      acc.c[k].x = buf[(s * 24 + 2 * k) * 32 + lane];
      acc.c[k].y = buf[(s * 24 + 2 * k + 1) * 32 + lane];
    }
  }

  const A hs = A(a.hop_scale);
#pragma unroll
  for (int k = 0; k < 12; k++) acc.c[k] = cscale(hs, acc.c[k]);

  if (a.local_mode != LOC_NONE && valid) {
    // M5op x at s = alpha x_s + beta (P- x_{s+1} + P+ x_{s-1});
    // M5op^dag x at s = alpha x_s + beta (P+ x_{s+1} + P- x_{s-1});
    // x_{Ls} = -mf x_0, x_{-1} = -mf x_{Ls-1}.
    Spinor<A> x0, xu, xd;
    load_spinor<P>(x0, a.in2, a.Vp, site, s);
    load_spinor<P>(xu, a.in2, a.Vp, site, s + 1 < LS ? s + 1 : 0);
    load_spinor<P>(xd, a.in2, a.Vp, site, s > 0 ? s - 1 : LS - 1);
    const A fu = (s + 1 < LS) ? A(1) : A(-a.mf);
    const A fd = (s > 0) ? A(1) : A(-a.mf);
    const A la = A(a.l_alpha), lb = A(a.l_beta);
    const bool dagm = (a.local_mode == LOC_M5DAG);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const bool plus = k < 6;
      const bool from_up = dagm ? plus : !plus;
      const cx<A> nb = from_up ? cscale(fu, xu.c[k]) : cscale(fd, xd.c[k]);
      acc.c[k].x += la * x0.c[k].x + lb * nb.x;
      acc.c[k].y += la * x0.c[k].y + lb * nb.y;
    }
  }

  double nrm = 0.0;
  if (a.epi == EPI_CG_R) {
    const A al = A(a.alpha[blockIdx.x / a.seg_cps]);
    Spinor<A> rr;
    load_spinor<P>(rr, a.r, a.Vp, site, s);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      rr.c[k].x -= al * acc.c[k].x;
      rr.c[k].y -= al * acc.c[k].y;
    }
    store_spinor<P>(a.r, a.Vp, site, s, rr);
    // the norm of what was stored (rounded to the storage precision)
    Spinor<A> back = rr;
    round_to_storage<P>(back);
#pragma unroll
    for (int k = 0; k < 12; k++)
      nrm += (double)back.c[k].x * back.c[k].x + (double)back.c[k].y * back.c[k].y;
  } else {
    store_spinor<P>(a.out, a.Vp, site, s, acc);
    if (a.epi == EPI_NORM) {
#pragma unroll
      for (int k = 0; k < 12; k++)
        nrm += (double)acc.c[k].x * acc.c[k].x + (double)acc.c[k].y * acc.c[k].y;
    }
  }
  if (a.epi != EPI_STORE) {
    double v[1] = {nrm};
    grid_reduce<1>(a.red, v, red_scratch);
  }
}

template <int P>
size_t stage_smem_bytes(int Ls, bool post) {
  return post ? (size_t)(Ls * 24 * 32 + 2 * Ls * Ls) * sizeof(typename Prec<P>::acc) : 0;
}

}  // namespace dwf
