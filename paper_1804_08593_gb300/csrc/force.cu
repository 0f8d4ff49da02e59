// Pseudofermion action S = phi^dag (Mpc^dag Mpc)^-1 phi and its gradient with respect to the
// links (PyTorch complex convention dS/dRe U + i dS/dIm U).
//
// With X = A^-1 phi, Y = Mpc X, V = D+ X (even), W = D+ M5op^-1 Dh_oe V (odd) and
// Z = M5op^-dag D+^dag Dh^dag_oe Y (odd):  dS = 1/2 Re(<Y, dDh W> + <Z, dDh V>).
// U_mu(x) enters Dh as (1 - gamma_mu) U_mu(x) b(x+mu) at output x and as
// (1 + gamma_mu) U_mu(x)^dag b(x) at output x+mu, so for full-lattice fields a, b the gradient
// of Re <a, Dh b> at link (x, mu) is
//   sum_s sum_spin [(1 - gamma_mu) a(x,s)] b(x+mu,s)^dag + b(x,s) [(1 + gamma_mu) a(x+mu,s)]^dag.
// For an even site x only Y(x), V(x) and W(x+mu), Z(x+mu) are non-zero; for an odd site only
// Z(x), W(x) and V(x+mu), Y(x+mu).  One thread computes the 3x3 gradient of one link.
#include <cmath>

#include "engine.h"

namespace dwf {

// out = (1 + sgn gamma_mu) in  (chiral basis, same factorisation as the hopping term)
template <int MU>
__device__ __forceinline__ void project(Spinor<double>& out, const Spinor<double>& in,
                                        double sgn) {
  for (int a = 0; a < 3; a++) {
    const cx<double> p0 = in.c[a], p1 = in.c[3 + a], p2 = in.c[6 + a], p3 = in.c[9 + a];
    cx<double> b0, b1;
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
    const cx<double> h0 = {p0.x + sgn * b0.x, p0.y + sgn * b0.y};
    const cx<double> h1 = {p1.x + sgn * b1.x, p1.y + sgn * b1.y};
    cx<double> l0, l1;
    if constexpr (MU == 0) {
      l0 = mul_i(h1);
      l1 = mul_i(h0);
    } else if constexpr (MU == 1) {
      l0 = h1;
      l1 = {-h0.x, -h0.y};
    } else if constexpr (MU == 2) {
      l0 = mul_i(h0);
      l1 = mul_i(h1); l1 = {-l1.x, -l1.y};
    } else {
      l0 = h0;
      l1 = h1;
    }
    out.c[a] = h0;
    out.c[3 + a] = h1;
    out.c[6 + a] = {sgn * l0.x, sgn * l0.y};
    out.c[9 + a] = {sgn * l1.x, sgn * l1.y};
  }
}

// acc[a][b] += sum_spin u_spin,a conj(v_spin,b)
__device__ __forceinline__ void outer_acc(cx<double> (&acc)[9], const Spinor<double>& u,
                                          const Spinor<double>& v) {
  for (int sp = 0; sp < 4; sp++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        const cx<double> x = u.c[sp * 3 + a], y = v.c[sp * 3 + b];
        acc[a * 3 + b].x += x.x * y.x + x.y * y.y;
        acc[a * 3 + b].y += x.y * y.x - x.x * y.y;
      }
}

struct ForceArgs {
  const void *Ye, *Ve, *Wo, *Zo;  // FP64 internal fields
  const uint32_t* nbr[2];
  const int* lex[2];
  double2* out;                    // caller layout [V][4][9]
  long Vp;
  int Ls;
};

template <int MU>
__device__ void force_link(const ForceArgs& a, int p, long idx) {
  // x even: (1-g) Y(x) W(x+mu)^dag + V(x) [(1+g) Z(x+mu)]^dag
  // x odd : (1-g) Z(x) V(x+mu)^dag + W(x) [(1+g) Y(x+mu)]^dag
  const void* A = p == 0 ? a.Ye : a.Zo;
  const void* B = p == 0 ? a.Wo : a.Ve;
  const void* C = p == 0 ? a.Ve : a.Wo;
  const void* D = p == 0 ? a.Zo : a.Ye;
  const long nidx = (long)(a.nbr[p][(long)(2 * MU) * a.Vp + idx] & NBR_IDX);
  cx<double> acc[9];
  for (int k = 0; k < 9; k++) acc[k] = {0.0, 0.0};
  for (int s = 0; s < a.Ls; s++) {
    Spinor<double> x, y, px;
    load_spinor<P64>(x, A, a.Vp, idx, s);
    load_spinor<P64>(y, B, a.Vp, nidx, s);
    project<MU>(px, x, -1.0);
    outer_acc(acc, px, y);
    load_spinor<P64>(x, C, a.Vp, idx, s);
    load_spinor<P64>(y, D, a.Vp, nidx, s);
    project<MU>(px, y, 1.0);
    outer_acc(acc, x, px);
  }
  const long lx = a.lex[p][idx];
  double2* o = a.out + (lx * 4 + MU) * 9;
  for (int k = 0; k < 9; k++) o[k] = make_double2(0.5 * acc[k].x, 0.5 * acc[k].y);
}

__global__ void force_kernel(const ForceArgs a) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y, p = blockIdx.z;
  if (idx >= a.Vp || a.lex[p][idx] < 0) return;
  switch (mu) {
    case 0: force_link<0>(a, p, idx); break;
    case 1: force_link<1>(a, p, idx); break;
    case 2: force_link<2>(a, p, idx); break;
    default: force_link<3>(a, p, idx);
  }
}


}  // namespace dwf

using namespace dwf;

// Solve to tol into a workspace buffer when the caller gives no X.
static dwf_status solution(dwf_t h, Layout* lay, const void* dphi, const void* X, double tol,
                           const void** dX) {
  const size_t ub = (size_t)h->Ls * (lay->g.V / 2) * 12 * 16;
  if (X) {
    void* p;
    DWF_TRY(stage_buffer(h, "force_X", X, ub, true, &p));
    *dX = p;
    return DWF_OK;
  }
  void* p;
  DWF_TRY(h->ws->get("force_X", ub, &p));
  DWF_CUDA(cudaMemsetAsync(p, 0, ub, h->stream));
  dwf_stats st{};
  dwf_status s = dwf_cg(h, dphi, p, tol, 1000000, DWF_F64, &st);
  if (s != DWF_OK) return s;
  *dX = p;
  return DWF_OK;
}

extern "C" dwf_status dwf_force(dwf_t h, const void* phi, const void* X, void* dSdU,
                                double tol) {
  if (!h || !phi || !dSdU) return set_error(DWF_ERR_ARG, "null argument");
  Layout* lay;
  DWF_TRY(get_layout(h, h->dims, &lay));
  const Geom& g = lay->g;
  const size_t ub = (size_t)h->Ls * (g.V / 2) * 12 * 16;
  void* dphi;
  DWF_TRY(stage_buffer(h, "force_phi", phi, ub, true, &dphi));
  const void* dX;
  DWF_TRY(solution(h, lay, dphi, X, tol, &dX));
  OpEngine E;
  DWF_TRY(E.init(h, lay, P64, false));
  const size_t fb = field_bytes(g, P64);
  void *x, *u, *w, *y, *z;
  DWF_TRY(h->ws->get("force_x", fb, &x));
  DWF_TRY(h->ws->get("force_u", fb, &u));
  DWF_TRY(h->ws->get("force_w", fb, &w));
  DWF_TRY(h->ws->get("force_y", fb, &y));
  DWF_TRY(h->ws->get("force_z", fb, &z));
  DWF_TRY(pack_even(h, lay, dX, x, P64, 1.0));
  // Y = Mpc X; the first stage leaves W = D+ M5op^-1 Dh_oe D+ X in w and D+ X in u
  DWF_TRY(E.mpc(x, u, w, y, EPI_STORE, RedArgs{}, nullptr));
  const void* V = x;
  if (!E.trivial()) {
    V = u;
  } else if (h->b != 1.0) {
    // D+ = b: V = b X
    VopArgs a{};
    a.op = VOP_ZERO;
    a.y = u;
    a.Vp = g.Vp;
    a.Vhb = g.Vhb;
    a.Vhb_pad = g.Vhb_pad;
    DWF_CUDA(launch_vop(P64, P64, a, h->Ls, h->stream));
    a.op = VOP_AXPY;
    a.x = x;
    a.sa = h->b;
    DWF_CUDA(launch_vop(P64, P64, a, h->Ls, h->stream));
    V = u;
  }
  // Z = M5op^-dag D+^dag Dh^dag_oe Y: first stage of Mpc^dag
  {
    StageArgs a = E.base(1);
    a.in = y;
    a.out = z;
    a.post = h->mats.d_m5idpt[0];
    a.epi = EPI_STORE;
    DWF_TRY(E.launch(a, true));
  }
  void* dout;
  const size_t lb = (size_t)g.V * 4 * 9 * 16;
  DWF_TRY(stage_buffer(h, "force_out", dSdU, lb, false, &dout));
  ForceArgs fa{};
  fa.Ye = y;
  fa.Ve = V;
  fa.Wo = w;
  fa.Zo = z;
  fa.nbr[0] = lay->nbr[0];
  fa.nbr[1] = lay->nbr[1];
  fa.lex[0] = lay->lex[0];
  fa.lex[1] = lay->lex[1];
  fa.out = reinterpret_cast<double2*>(dout);
  fa.Vp = g.Vp;
  fa.Ls = h->Ls;
  dim3 grid((unsigned)((g.Vp + 127) / 128), 4, 2);
  force_kernel<<<grid, 128, 0, h->stream>>>(fa);
  DWF_CUDA(cudaGetLastError());
  return finish_output(h, dSdU, dout, lb);
}

extern "C" dwf_status dwf_action(dwf_t h, const void* phi, const void* X, double tol, double* S) {
  if (!h || !phi || !S) return set_error(DWF_ERR_ARG, "null argument");
  Layout* lay;
  DWF_TRY(get_layout(h, h->dims, &lay));
  const Geom& g = lay->g;
  const size_t ub = (size_t)h->Ls * (g.V / 2) * 12 * 16;
  void* dphi;
  DWF_TRY(stage_buffer(h, "force_phi", phi, ub, true, &dphi));
  const void* dX;
  DWF_TRY(solution(h, lay, dphi, X, tol, &dX));
  OpEngine E;
  DWF_TRY(E.init(h, lay, P64, false));
  const size_t fb = field_bytes(g, P64);
  void *x, *f, *u, *t, *y;
  double* d;
  DWF_TRY(h->ws->get("force_x", fb, &x));
  DWF_TRY(h->ws->get("force_f", fb, &f));
  DWF_TRY(h->ws->get("force_u", fb, &u));
  DWF_TRY(h->ws->get("force_w", fb, &t));
  DWF_TRY(h->ws->get("force_y", fb, &y));
  DWF_TRY(h->ws->get("force_d", 4 * sizeof(double), (void**)&d));
  DWF_TRY(pack_even(h, lay, dX, x, P64, 1.0));
  DWF_TRY(pack_even(h, lay, dphi, f, P64, 1.0));
  // S = Re(2 <phi, X> - ||Mpc X||^2): equals phi^dag A^-1 phi at the exact solution, with an
  // error quadratic in the solve residual.
  DWF_TRY(E.mpc(x, u, t, y, EPI_NORM, E.red(FIN_STORE, d), nullptr));
  VopArgs a{};
  a.op = VOP_DOT;
  a.x = f;
  a.y = x;
  a.Vp = g.Vp;
  a.Vhb = g.Vhb;
  a.Vhb_pad = g.Vhb_pad;
  a.red = E.red(FIN_STORE, d + 1);
  DWF_CUDA(launch_vop(P64, P64, a, h->Ls, h->stream));
  double hv[2];
  DWF_CUDA(cudaMemcpyAsync(hv, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  *S = 2.0 * hv[1] - hv[0];
  return DWF_OK;
}
