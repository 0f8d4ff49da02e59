// Krylov solvers on A = Mpc^dag Mpc (Sec. 2.2, Eq. 3):
//   * CG with device-resident scalars and a device stop flag, in FP64 or in a low precision
//     with FP64 reliable updates;
//   * multisplitting preconditioned CG (Sec. 2.3): the preconditioner M = sum_s A_s (Eq. 5)
//     applied as l local CG iterations per lattice block from a zero guess (Eq. 4), all
//     blocks at once with block-local reductions, in FP16/BF16/FP32/FP64 storage; the outer
//     CG in FP32 (FP64 reliable updates) or FP64.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "engine.h"

namespace dwf {

// Reliable updates: the low-precision iteration hands its iterate to the FP64 solution and
// restarts from the FP64 true residual b - A x once its own residual has dropped by delta
// (DWF_RU_DELTA overrides 0.1; values outside (0, 1) are ignored).
static double ru_delta() {
  const char* e = getenv("DWF_RU_DELTA");
  const double d = e ? atof(e) : 0.1;
  return (d > 0.0 && d < 1.0) ? d : 0.1;
}

// Device scalar slots of one solve.
enum Slot {
  S_RHO = 0,    // CG: ||r||^2 ; PCG: <r, z>
  S_ALPHA = 1,
  S_BETA = 2,
  S_PAP = 3,    // <p, A p> = ||Mpc p||^2
  S_RR = 4,     // ||r||^2 (PCG)
  S_STOP2 = 5,  // stop threshold on ||r||^2
  S_TMP = 6,
  S_RZNEW = 7,
  S_NSLOT = 16
};
enum Flag { F_CONV = 0, F_STOP = 1, F_ITER = 2, F_NFLAG = 8 };

// ---------------------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------------------
static dwf_status vop(const OpEngine& E, int op, const void* x, void* y, RedArgs red = {},
                      double sa = 1.0, const double* ap = nullptr, int prec_x = -1) {
  VopArgs a{};
  a.op = op;
  a.x = x;
  a.y = y;
  a.Vp = E.g().Vp;
  a.Vhb = E.g().Vhb;
  a.Vhb_pad = E.g().Vhb_pad;
  a.sa = sa;
  a.ap = ap;
  a.red = red;
  ProfScope ps(&E.h->prof, E.h->stream, "vector_ops", 2.0 * field_bytes(E.g(), E.prec), 0.0);
  DWF_CUDA(launch_vop(E.prec, prec_x < 0 ? E.prec : prec_x, a, E.h->Ls, E.h->stream));
  return DWF_OK;
}

// out (Eout's layout and precision) = f * in, f = num or sqrt(num / *den) (inverted if asked);
// in_map: in is in another site order (out site i reads in site in_map[i], stride vp_in)
// out3: also u = D+ out (the Moebius pre-op of what was stored), in the same pass
static dwf_status cast(const OpEngine& Eout, int pin, const void* in, void* out, double num,
                       const double* den, int invert, const void* dotv, RedArgs red,
                       void* out2 = nullptr, const int* in_map = nullptr, long vp_in = 0,
                       void* out3 = nullptr) {
  CastArgs a{};
  a.in = in;
  a.out = out;
  a.in_map = in_map;
  a.Vp_in = vp_in;
  a.out3 = out3;
  a.db = Eout.h->b;
  a.dc = Eout.h->c;
  a.mf = Eout.h->mf;
  a.dbf = (float)a.db;
  a.dcf = (float)a.dc;
  a.mff = (float)a.mf;
  a.Vp = Eout.g().Vp;
  a.Vhb = Eout.g().Vhb;
  a.Vhb_pad = Eout.g().Vhb_pad;
  a.num = num;
  a.den = den;
  a.invert = invert;
  a.dotv = dotv;
  a.out2 = out2;
  a.red = red;
  ProfScope ps(&Eout.h->prof, Eout.h->stream, "cast",
               field_bytes(Eout.g(), pin) +
                   field_bytes(Eout.g(), Eout.prec) *
                       ((out ? 1 : 0) + (out2 ? 1 : 0) + (out3 ? 1 : 0)) +
                   (dotv ? field_bytes(Eout.g(), Eout.prec) : 0),
               0.0);
  DWF_CUDA(launch_cast(pin, Eout.prec, a, Eout.h->Ls, Eout.h->stream));
  return DWF_OK;
}

// x/p/u update: bytes = reads of p (+x, r) and writes of x (+p, u).
static dwf_status vec(const OpEngine& E, const VecArgs& va, double zbytes = 0.0) {
  const double f = (double)field_bytes(E.g(), E.prec);
  // p read; x read and written; r (or the preconditioner output) read and p written; u written
  const double rb = va.z_src ? zbytes : f;
  const double bytes = f * (1 + 2 * va.do_x + va.do_p + va.do_u) + (va.do_p ? rb : 0.0);
  char name[32];
  snprintf(name, sizeof(name), "cg_update_%s", prec_name(E.prec));
  ProfScope ps(&E.h->prof, E.h->stream, name, bytes, 0.0);
  DWF_CUDA(launch_vec(E.prec, va, E.h->Ls, E.h->stream));
  return DWF_OK;
}

static dwf_status read_doubles(dwf_ctx* h, const double* dev, int n, double* out) {
  DWF_CUDA(cudaMemcpyAsync(h->h_pinned, dev, n * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  memcpy(out, h->h_pinned, n * sizeof(double));
  return DWF_OK;
}

static dwf_status read_ints(dwf_ctx* h, const int* dev, int n, int* out) {
  DWF_CUDA(cudaMemcpyAsync(h->h_pinned, dev, n * sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  memcpy(out, h->h_pinned, n * sizeof(int));
  return DWF_OK;
}

static dwf_status write_doubles(dwf_ctx* h, double* dev, const double* v, int n) {
  // pageable source: the copy is staged before the call returns
  DWF_CUDA(cudaMemcpyAsync(dev, v, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  return DWF_OK;
}

// r = b - A x in FP64 (x nullptr: r = b), returns ||r||^2 on the host.
static dwf_status true_residual(const OpEngine& E64, const void* b, const void* x, void* r,
                                void* t1, void* t2, void* t3, double* dsc, double* rr) {
  if (x) {
    DWF_TRY(E64.mpc(x, t1, t2, t3, EPI_STORE, RedArgs{}, nullptr));
    DWF_TRY(E64.mpcdag(t3, t2, r, EPI_STORE, nullptr, nullptr, RedArgs{}, nullptr));
    DWF_TRY(vop(E64, VOP_XMY_NORM, b, r, E64.red(FIN_STORE, dsc + S_TMP)));
  } else {
    DWF_TRY(vop(E64, VOP_COPY, b, r));
    DWF_TRY(vop(E64, VOP_NORM, r, nullptr, E64.red(FIN_STORE, dsc + S_TMP)));
  }
  return read_doubles(E64.h, dsc + S_TMP, 1, rr);
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double seconds() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

static void stats_init(dwf_stats* st) {
  if (!st) return;
  st->iterations = st->inner_iterations = st->reliable_updates = 0;
  st->operator_applications = 0;
  st->true_residual = 0.0;
  st->seconds = 0.0;
  st->history_len = 0;
}

// ---------------------------------------------------------------------------------------
// CG with reliable updates.
// ---------------------------------------------------------------------------------------
struct CGVectors {
  void *x, *p, *r, *u, *t, *y, *s;
};

// One CG iteration on the low-precision engine E; all scalars stay on the device.
static dwf_status cg_iteration(const OpEngine& E, const CGVectors& v, double* dsc, int* dfl,
                               double* hist, double* curv, int hist_cap) {
  const int* stop = dfl + F_STOP;
  RedArgs ra = E.red(FIN_ALPHA, dsc + S_PAP);
  ra.rho = dsc + S_RHO;
  ra.alpha = dsc + S_ALPHA;
  ra.hist = curv;   // <p, A p> of this iteration (Lanczos coefficients)
  ra.hist_idx = dfl + F_ITER;
  ra.hist_cap = curv ? hist_cap : 0;
  DWF_TRY(E.mpc(v.p, v.u, v.t, v.y, EPI_NORM, ra, stop, true));
  RedArgs rb = E.red(FIN_BETA, nullptr);
  rb.rho = dsc + S_RHO;
  rb.beta = dsc + S_BETA;
  rb.stop2 = dsc + S_STOP2;
  rb.conv = dfl + F_CONV;
  rb.hist = hist;
  rb.hist_idx = dfl + F_ITER;
  rb.hist_cap = hist_cap;
  DWF_TRY(E.mpcdag(v.y, v.s, nullptr, EPI_CG_R, v.r, dsc + S_ALPHA, rb, stop));
  VecArgs va{};
  va.x = v.x;
  va.p = v.p;
  va.r = v.r;
  va.u = v.u;
  va.Vp = E.g().Vp;
  va.Vhb = E.g().Vhb;
  va.Vhb_pad = E.g().Vhb_pad;
  va.alpha = dsc + S_ALPHA;
  va.beta = dsc + S_BETA;
  va.seg_cps = E.seg_cps;
  va.do_x = 1;
  va.do_p = 1;
  va.do_u = E.trivial() ? 0 : 1;
  va.db = E.h->b;
  va.dc = E.h->c;
  va.mf = E.h->mf;
  va.stop = stop;
  va.red.counter = E.h->red_counter;
  va.stop_out = dfl + F_STOP;
  va.conv_in = dfl + F_CONV;
  va.iter = dfl + F_ITER;
  return vec(E, va);
}

static dwf_status run_cg(dwf_ctx* h, Layout* lay, const void* b_c128, void* x_c128, bool x0,
                         double tol, int maxit, int prec, dwf_stats* stats) {
  Timer timer;
  stats_init(stats);
  const Geom& g = lay->g;
  OpEngine E64, E;
  DWF_TRY(E64.init(h, lay, P64, false));
  DWF_TRY(E.init(h, lay, prec, false));
  const size_t f64 = field_bytes(g, P64), flo = field_bytes(g, prec);
  void *b64, *x64, *r64, *t1, *t2, *t3;
  DWF_TRY(h->ws->get("cg_b64", f64, &b64));
  DWF_TRY(h->ws->get("cg_x64", f64, &x64));
  DWF_TRY(h->ws->get("cg_r64", f64, &r64));
  DWF_TRY(h->ws->get("cg_t1", f64, &t1));
  DWF_TRY(h->ws->get("cg_t2", f64, &t2));
  DWF_TRY(h->ws->get("cg_t3", f64, &t3));
  CGVectors v;
  DWF_TRY(h->ws->get("cg_x", flo, &v.x));
  DWF_TRY(h->ws->get("cg_p", flo, &v.p));
  DWF_TRY(h->ws->get("cg_r", flo, &v.r));
  DWF_TRY(h->ws->get("cg_u", flo, &v.u));
  DWF_TRY(h->ws->get("cg_t", flo, &v.t));
  DWF_TRY(h->ws->get("cg_y", flo, &v.y));
  DWF_TRY(h->ws->get("cg_s", flo, &v.s));
  double* dsc;
  int* dfl;
  double* dhist = nullptr;
  double* dcurv = nullptr;
  DWF_TRY(h->ws->get("cg_scal", S_NSLOT * sizeof(double), (void**)&dsc));
  DWF_TRY(h->ws->get("cg_flag", F_NFLAG * sizeof(int), (void**)&dfl));
  const int hcap = (stats && stats->history && stats->history_capacity > 0)
                       ? stats->history_capacity : 0;
  if (hcap) DWF_TRY(h->ws->get("cg_hist", (size_t)hcap * sizeof(double), (void**)&dhist));
  if (hcap && stats->curvature_history)
    DWF_TRY(h->ws->get("cg_curv", (size_t)hcap * sizeof(double), (void**)&dcurv));

  DWF_TRY(pack_even(h, lay, b_c128, b64, P64, 1.0));
  if (x0) DWF_TRY(pack_even(h, lay, x_c128, x64, P64, 1.0));
  else DWF_TRY(vop(E64, VOP_ZERO, nullptr, x64));

  double bb, rr;
  DWF_TRY(vop(E64, VOP_NORM, b64, nullptr, E64.red(FIN_STORE, dsc + S_TMP)));
  DWF_TRY(read_doubles(h, dsc + S_TMP, 1, &bb));
  if (!(bb > 0.0) || !std::isfinite(bb)) {
    if (bb == 0.0) {  // zero source: zero solution
      DWF_TRY(vop(E64, VOP_ZERO, nullptr, x64));
      DWF_TRY(unpack_even(h, lay, x64, P64, x_c128, 1.0));
      DWF_CUDA(cudaStreamSynchronize(h->stream));
      if (stats) stats->seconds = timer.seconds();
      return DWF_OK;
    }
    return set_error(DWF_ERR_BREAKDOWN, "source norm is not finite");
  }
  DWF_TRY(true_residual(E64, b64, x0 ? x64 : nullptr, r64, t1, t2, t3, dsc, &rr));
  if (stats) stats->operator_applications += x0 ? 1 : 0;

  const double delta = (prec == P64) ? 0.0 : ru_delta();
  const bool scaled = (prec == P16 || prec == PB16);
  const double nreal = 24.0 * h->Ls * (double)(g.V / 2);
  const double tol2 = tol * tol * bb;
  int iters = 0, total_hist = 0;
  std::vector<double> hist_scale;  // scale of each recorded history entry
  double scale = 1.0;
  bool restart_p = true;
  // A low-precision cycle ends when its residual has dropped by delta, after `cap`
  // iterations (16-bit CG loses accuracy long before that when kappa * eps ~ 1), or when
  // its residual grows by more than 1e6 (divergence); the last two restart p = r.
  const int cap = (prec == P16 || prec == PB16) ? 200 : (1 << 30);
  dwf_status status = DWF_OK;
  while (true) {
    if (rr <= tol2) break;
    if (!std::isfinite(rr)) {
      status = set_error(DWF_ERR_BREAKDOWN, "residual is not finite");
      break;
    }
    if (iters >= maxit) {
      status = set_error(DWF_ERR_NOT_CONVERGED, "maximum number of iterations reached");
      break;
    }
    // (re)start a low-precision cycle from the FP64 residual
    const double new_scale = scaled ? std::sqrt(nreal / rr) : 1.0;
    DWF_TRY(cast(E, P64, r64, v.r, new_scale, nullptr, 0, nullptr,
                 E.red(FIN_STORE, dsc + S_RHO)));
    DWF_TRY(vop(E, VOP_ZERO, nullptr, v.x));
    if (restart_p) {
      DWF_TRY(vop(E, VOP_COPY, v.r, v.p));
      if (!E.trivial()) DWF_TRY(E.dplus(v.p, v.u, nullptr));
    } else if (new_scale != scale) {
      // keep the search direction, expressed in the new scale
      const double f = new_scale / scale;
      DWF_TRY(vop(E, VOP_AXPY, v.p, v.p, RedArgs{}, f - 1.0));
      if (!E.trivial()) DWF_TRY(vop(E, VOP_AXPY, v.u, v.u, RedArgs{}, f - 1.0));
    }
    scale = new_scale;
    restart_p = false;
    const double rho0 = scale * scale * rr;
    const double stop2 = scale * scale * std::max(delta * delta * rr, tol2);
    double hs[2] = {stop2, 0.0};
    DWF_TRY(write_doubles(h, dsc + S_STOP2, hs, 1));
    DWF_CUDA(cudaMemsetAsync(dfl, 0, F_NFLAG * sizeof(int), h->stream));
    int chunk = 8, done_cycle = 0;
    int fl[F_NFLAG] = {0};
    bool finite_cycle = true;
    while (true) {
      const int n = std::min(chunk, maxit - iters - done_cycle);
      if (n <= 0) break;
      for (int k = 0; k < n; k++)
        DWF_TRY(cg_iteration(E, v, dsc, dfl, dhist ? dhist + total_hist : nullptr,
                             dcurv ? dcurv + total_hist : nullptr,
                             dhist ? hcap - total_hist : 0));
      double rho;
      DWF_TRY(read_ints(h, dfl, F_NFLAG, fl));
      DWF_TRY(read_doubles(h, dsc + S_RHO, 1, &rho));
      done_cycle = fl[F_ITER];
      if (!std::isfinite(rho)) {
        finite_cycle = false;
        restart_p = true;
        break;
      }
      if (fl[F_STOP]) break;
      if (done_cycle >= cap || rho > 1e6 * rho0) {
        restart_p = true;
        break;
      }
      chunk = std::min(chunk * 2, 64);
    }
    iters += done_cycle;
    total_hist += done_cycle;
    hist_scale.resize(total_hist, scale);
    if (stats) stats->operator_applications += done_cycle;
    // reliable update: x64 += x / scale, r64 = b - A x64
    if (finite_cycle)
      DWF_TRY(vop(E64, VOP_ADD_CAST, v.x, x64, RedArgs{}, 1.0 / scale, nullptr, prec));
    DWF_TRY(true_residual(E64, b64, x64, r64, t1, t2, t3, dsc, &rr));
    if (stats) {
      stats->reliable_updates++;
      stats->operator_applications++;
    }
  }
  DWF_TRY(unpack_even(h, lay, x64, P64, x_c128, 1.0));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  if (stats) {
    stats->iterations = iters;
    stats->true_residual = std::sqrt(rr / bb);
    if (hcap) {
      const int n = std::min(total_hist, hcap);
      std::vector<double> hv(n);
      if (n) DWF_CUDA(cudaMemcpy(hv.data(), dhist, n * sizeof(double), cudaMemcpyDeviceToHost));
      // hist holds the low-precision ||r||^2 in scaled units; report relative norms
      for (int i = 0; i < n; i++) stats->history[i] = std::sqrt(hv[i] / bb) / hist_scale[i];
      stats->history_len = n;
      if (dcurv && n) {
        DWF_CUDA(cudaMemcpy(hv.data(), dcurv, n * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; i++)
          stats->curvature_history[i] = hv[i] / (bb * hist_scale[i] * hist_scale[i]);
      }
    }
    stats->seconds = timer.seconds();
  }
  return status;
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_cg(dwf_t h, const void* phi, void* x, double tol, int maxit,
                             dwf_prec prec, dwf_stats* stats) {
  if (!h || !phi || !x) return set_error(DWF_ERR_ARG, "null argument");
  if (!(tol > 0.0) || maxit < 0) return set_error(DWF_ERR_ARG, "bad tolerance or maxit");
  if ((int)prec < 0 || (int)prec > 3) return set_error(DWF_ERR_ARG, "bad precision");
  Layout* lay;
  DWF_TRY(get_layout(h, h->dims, &lay));
  const size_t ub = (size_t)h->Ls * (lay->g.V / 2) * 12 * 16;
  void *db, *dx;
  DWF_TRY(stage_buffer(h, "io_phi", phi, ub, true, &db));
  DWF_TRY(stage_buffer(h, "io_x", x, ub, true, &dx));
  dwf_status st = run_cg(h, lay, db, dx, true, tol, maxit, (int)prec, stats);
  if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
  dwf_status st2 = finish_output(h, x, dx, ub);
  return st2 != DWF_OK ? st2 : st;
}

// ---------------------------------------------------------------------------------------
// Multisplitting preconditioned CG.
// ---------------------------------------------------------------------------------------
namespace dwf {

// beta = (<r, z> - <r_old, z>) / rho_old, rho = <r, z>   (Polak-Ribiere)
__global__ void pr_beta_kernel(double* d) {
  const double rz = d[S_RZNEW], rold_z = d[S_TMP], rho = d[S_RHO];
  d[S_BETA] = (rho > 0.0 && isfinite(rz)) ? (rz - rold_z) / rho : 0.0;
  d[S_RHO] = rz;
}

// Where the outer update reads z from when z is not stored: the local solution in its own
// site order and precision, with the scale that undoes the local solver's normalisation.
struct ZSrc {
  const void* src = nullptr;
  int prec = 0;
  const int* map = nullptr;
  long vp = 0;
  double num = 1.0;
  const double* den = nullptr;
  double bytes = 0.0;
};

struct InnerVectors {
  void *ri, *xi, *pi, *ui, *ti, *yi, *si;
  bool exact = false;
  OpEngine::ExactBufs eb{};
  SimdLocal* simd = nullptr;   // local solves in one persistent launch (else stage launches)
  int prec = 0;                // storage precision of the local solves
};

// Which local solver MSPCG uses: the persistent block-SIMD kernel or one launch per operator
// stage.  Default: persistent for FP32/FP16/BF16 local solves; stages for FP64, where the
// persistent kernel (one slice per thread, one CTA per SM at its register use) measured slower.
// DWF_LOCAL_SOLVER=persistent|stages forces one.
static bool use_simd_local(int inner) {
  const char* e = getenv("DWF_LOCAL_SOLVER");
  if (e && strcmp(e, "stages") == 0) return false;
  if (e && strcmp(e, "persistent") == 0) return true;
  return inner != P64;
}

static dwf_status precondition_stages(const OpEngine& Em, const OpEngine& Ei, const void* r,
                                      const InnerVectors& iv, double* dsc, double* blk, int nb,
                                      int l);

// The preconditioner step of the persistent local solver (the local solves' launch and the
// reductions that follow it) as a CUDA graph: captured once the solver's launch variant is
// decided (never while the per-launch profiler is on, whose events must be recorded per
// launch), then replayed by every later preconditioner call of the solve.  Every argument of
// the step (buffers, scalar slots, sizes) is the same on every call.  DWF_PRECOND_GRAPH=0
// issues the launches directly.
struct PcGraph {
  cudaGraphExec_t exec = nullptr;
  bool tried = false;
  ~PcGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

static bool pc_graph_enabled(dwf_ctx* h, const InnerVectors& iv) {
  const char* e = getenv("DWF_PRECOND_GRAPH");
  if (e && strcmp(e, "0") == 0) return false;
  if (h->prof.on || !iv.simd || !simd_variant_decided(iv.simd, iv.prec)) return false;
  // the legacy default stream cannot be captured: handles created without a stream launch
  // directly
  if (h->stream == nullptr || h->stream == cudaStreamLegacy) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess &&
         cs == cudaStreamCaptureStatusNone;
}

// z = M^-1 r approximated by l local CG iterations per block from a zero guess (Eqs. 4-5),
// with every block-local dot product reduced per block; then <r, z> (FR) or the
// Polak-Ribiere numerator is reduced and beta is finalised on the device.
// Non-flexible: z is not stored; zs tells the outer update where to read it, and <r, z> (for
// the Fletcher-Reeves beta) is reduced from the local solution directly.
static dwf_status precondition(const OpEngine& Em, const OpEngine& Ei, const void* r, void* z,
                               const InnerVectors& iv, double* dsc, double* blk, int nb, int l,
                               bool flexible, const void* rold, ZSrc& zs, PcGraph* pg) {
  const int ip = iv.prec;
  const bool scaled = (ip == P16 || ip == PB16);
  const double nreal = 24.0 * Em.h->Ls * (double)(Em.g().V / 2);
  // where the local solution lives: element order and stride, and its bytes
  const int* zmap = nullptr;
  long zvp = 0;
  double zbytes = 0.0;
  if (iv.simd) {
    zmap = iv.simd->inv;
    zvp = iv.simd->sB;
    zbytes = (double)Em.h->Ls * (double)iv.simd->sB * 24.0 * (double)real_bytes(ip);
  } else {
    DWF_TRY(precondition_stages(Em, Ei, r, iv, dsc, blk, nb, l));
    const bool remap = (Em.lay != Ei.lay);
    zmap = remap ? Ei.lay->cb_inv : nullptr;
    zvp = Ei.g().Vp;
    zbytes = (double)field_bytes(Ei.g(), Ei.prec);
  }
  // the device work after the stage-launched local solves, or all of it for the persistent
  // local solver
  auto issue = [&]() -> dwf_status {
    if (iv.simd) {
      const SimdFields F{iv.xi, iv.pi, iv.ui, iv.ri, iv.ti, iv.yi};
      DWF_TRY(simd_local_solve(Em.h, iv.simd, ip, l, r, Em.prec, Em.g().Vp,
                               scaled ? nreal : 1.0, scaled ? dsc + S_RR : nullptr, F));
    }
    if (!flexible) {
      RedArgs rz = Em.red(FIN_BETA, nullptr);
      rz.rho = dsc + S_RHO;
      rz.beta = dsc + S_BETA;
      DWF_TRY(cast(Em, ip, iv.xi, nullptr, scaled ? nreal : 1.0,
                   scaled ? dsc + S_RR : nullptr, 1, r, rz, nullptr, zmap, zvp));
    } else {
      DWF_TRY(cast(Em, ip, iv.xi, z, scaled ? nreal : 1.0, scaled ? dsc + S_RR : nullptr, 1,
                   r, Em.red(FIN_STORE, dsc + S_RZNEW), nullptr, zmap, zvp));
      DWF_TRY(vop(Em, VOP_DOT, rold, z, Em.red(FIN_STORE, dsc + S_TMP)));
      pr_beta_kernel<<<1, 1, 0, Em.h->stream>>>(dsc);
      DWF_CUDA(cudaGetLastError());
    }
    return DWF_OK;
  };
  cudaStream_t st = Em.h->stream;
  if (pg && pg->exec) {
    DWF_CUDA(cudaGraphLaunch(pg->exec, st));
  } else if (pg && !pg->tried && pc_graph_enabled(Em.h, iv)) {
    pg->tried = true;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return precondition(Em, Ei, r, z, iv, dsc, blk, nb, l, flexible, rold, zs, nullptr);
    }
    const dwf_status s_issue = issue();
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(st, &graph);
    cudaError_t e_inst = cudaErrorUnknown;
    if (s_issue == DWF_OK && e_end == cudaSuccess && graph)
      e_inst = cudaGraphInstantiate(&pg->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s_issue != DWF_OK) return s_issue;
    if (e_end != cudaSuccess || e_inst != cudaSuccess) {
      // not capturable here: nothing of the step ran, so issue it directly (and from now on)
      cudaGetLastError();
      pg->exec = nullptr;
      DWF_TRY(issue());
    } else {
      DWF_CUDA(cudaGraphLaunch(pg->exec, st));
    }
  } else {
    DWF_TRY(issue());
  }
  if (!flexible) {
    zs.src = iv.xi;
    zs.prec = ip;
    zs.map = zmap;
    zs.vp = zvp;
    zs.num = scaled ? nreal : 1.0;
    zs.den = scaled ? dsc + S_RR : nullptr;
    zs.bytes = zbytes;
  } else {
    zs = ZSrc{};
  }
  return DWF_OK;
}

// The local solves as one launch per operator stage and CG update, block-local reductions as
// CTA segments of the block-major site order; the solution is left in iv.xi.
static dwf_status precondition_stages(const OpEngine& Em, const OpEngine& Ei, const void* r,
                                      const InnerVectors& iv, double* dsc, double* blk, int nb,
                                      int l) {
  const bool scaled = (Ei.prec == P16 || Ei.prec == PB16);
  const double nreal = 24.0 * Em.h->Ls * (double)(Em.g().V / 2);
  double* rho_b = blk;
  double* alpha_b = blk + nb;
  double* beta_b = blk + 2 * nb;
  double* pap_b = blk + 3 * nb;
  // the outer vectors are in caller (lexicographic) site order, the local solves in block
  // order: the casts between the two gather through the layout's index maps
  const bool remap = (Em.lay != Ei.lay);
  DWF_TRY(cast(Ei, Em.prec, r, iv.ri, scaled ? nreal : 1.0, scaled ? dsc + S_RR : nullptr, 0,
               nullptr, Ei.red(FIN_STORE, rho_b), iv.pi, remap ? Ei.lay->cb_even : nullptr,
               Em.g().Vp, Ei.trivial() ? nullptr : iv.ui));
  DWF_TRY(vop(Ei, VOP_ZERO, nullptr, iv.xi));
  double* papx_b = blk + 4 * nb;
  for (int k = 0; k < l; k++) {
    // the last local iteration needs only ||Mpc p||^2 (for alpha), not Mpc p itself
    const bool last = (k + 1 == l);
    if (iv.exact) {
      DWF_TRY(Ei.exact_mpc(iv.pi, iv.ui, iv.eb, papx_b, rho_b, alpha_b, nullptr, !last));
    } else {
      RedArgs ra = Ei.red(FIN_ALPHA, pap_b);
      ra.rho = rho_b;
      ra.alpha = alpha_b;
      DWF_TRY(Ei.mpc(iv.pi, iv.ui, iv.ti, iv.yi, last ? EPI_NORM_ONLY : EPI_NORM, ra, nullptr,
                     true));
    }
    VecArgs va{};
    va.x = iv.xi;
    va.p = iv.pi;
    va.r = iv.ri;
    va.u = iv.ui;
    va.Vp = Ei.g().Vp;
    va.Vhb = Ei.g().Vhb;
    va.Vhb_pad = Ei.g().Vhb_pad;
    va.alpha = alpha_b;
    va.beta = beta_b;
    va.seg_cps = Ei.seg_cps;
    va.do_x = 1;
    va.db = Ei.h->b;
    va.dc = Ei.h->c;
    va.mf = Ei.h->mf;
    if (k + 1 < l) {
      RedArgs rb = Ei.red(FIN_BETA, nullptr);
      rb.rho = rho_b;
      rb.beta = beta_b;
      if (iv.exact)
        DWF_TRY(Ei.exact_mpcdag_cg(iv.eb, iv.ri, alpha_b, rb, nullptr));
      else
        DWF_TRY(Ei.mpcdag(iv.yi, iv.si, nullptr, EPI_CG_R, iv.ri, alpha_b, rb, nullptr));
      va.do_p = 1;
      va.do_u = Ei.trivial() ? 0 : 1;
    }
    DWF_TRY(vec(Ei, va));
  }
  return DWF_OK;
}

// lay: the block layout of the local solves; layL: the caller (lexicographic) order of the
// outer iteration, whose hops stay local in memory (the block order scatters them)
static dwf_status run_mspcg(dwf_ctx* h, Layout* lay, Layout* layL, int l, int inner,
                            int middle, bool flex, bool exact, const void* b_c128, void* x_c128,
                            double tol, int maxit, dwf_stats* stats) {
  Timer timer;
  stats_init(stats);
  const Geom& g = layL->g;     // outer vectors
  const Geom& gb = lay->g;     // local solves
  const bool simd = use_simd_local(inner);
  long max_ctas = std::max(g.Vp, gb.Vp) / 32;
  if (exact && !simd) {
    // before the engines pack links: packing also gathers the halo copies
    DWF_TRY(ensure_halo(h, lay));
    max_ctas = std::max(max_ctas, lay->halo->He_tot / 32);
  }
  OpEngine E64, Em, Ei;
  DWF_TRY(E64.init(h, layL, P64, false));
  DWF_TRY(Em.init(h, layL, middle, false));
  if (!simd) DWF_TRY(Ei.init(h, lay, inner, true));
  DWF_TRY(ensure_reduction(h, max_ctas * 2 + 64, gb.nblocks + 64));
  const size_t f64 = field_bytes(g, P64), fm = field_bytes(g, middle), fi = field_bytes(gb, inner);
  void *b64, *x64, *r64, *t1, *t2, *t3;
  DWF_TRY(h->ws->get("ms_b64", f64, &b64));
  DWF_TRY(h->ws->get("ms_x64", f64, &x64));
  DWF_TRY(h->ws->get("ms_r64", f64, &r64));
  DWF_TRY(h->ws->get("ms_t1", f64, &t1));
  DWF_TRY(h->ws->get("ms_t2", f64, &t2));
  DWF_TRY(h->ws->get("ms_t3", f64, &t3));
  void *xm, *rm, *pm, *um, *tm, *ym, *sm, *zm, *rold = nullptr;
  DWF_TRY(h->ws->get("ms_xm", fm, &xm));
  DWF_TRY(h->ws->get("ms_rm", fm, &rm));
  DWF_TRY(h->ws->get("ms_pm", fm, &pm));
  DWF_TRY(h->ws->get("ms_um", fm, &um));
  DWF_TRY(h->ws->get("ms_tm", fm, &tm));
  DWF_TRY(h->ws->get("ms_ym", fm, &ym));
  DWF_TRY(h->ws->get("ms_sm", fm, &sm));
  DWF_TRY(h->ws->get("ms_zm", fm, &zm));
  if (flex) DWF_TRY(h->ws->get("ms_rold", fm, &rold));
  InnerVectors iv;
  iv.prec = inner;
  if (simd) {
    DWF_TRY(ensure_simd(h, lay, exact, &iv.simd));
    const size_t per = (size_t)h->Ls * 24 * real_bytes(inner);
    DWF_TRY(h->ws->get("ms_ri", per * iv.simd->sB, &iv.ri));
    DWF_TRY(h->ws->get("ms_xi", per * iv.simd->sB, &iv.xi));
    DWF_TRY(h->ws->get("ms_pi", per * iv.simd->sB, &iv.pi));
    DWF_TRY(h->ws->get("ms_ui", per * iv.simd->sB, &iv.ui));
    DWF_TRY(h->ws->get("ms_ti", per * iv.simd->sO, &iv.ti));
    DWF_TRY(h->ws->get("ms_yi", per * iv.simd->sE, &iv.yi));
    iv.si = nullptr;
  } else {
  DWF_TRY(h->ws->get("ms_ri", fi, &iv.ri));
  DWF_TRY(h->ws->get("ms_xi", fi, &iv.xi));
  DWF_TRY(h->ws->get("ms_pi", fi, &iv.pi));
  DWF_TRY(h->ws->get("ms_ui", fi, &iv.ui));
  DWF_TRY(h->ws->get("ms_ti", fi, &iv.ti));
  DWF_TRY(h->ws->get("ms_yi", fi, &iv.yi));
  DWF_TRY(h->ws->get("ms_si", fi, &iv.si));
  if (exact) {
    const Halo& H = *lay->halo;
    const size_t per_site = (size_t)h->Ls * 24 * real_bytes(inner);
    iv.exact = true;
    iv.eb.t_int = iv.ti;
    iv.eb.y_int = iv.yi;
    iv.eb.s_int = iv.si;
    DWF_TRY(h->ws->get("ms_th", per_site * H.Ho_tot, &iv.eb.t_halo));
    DWF_TRY(h->ws->get("ms_sh", per_site * H.Ho_tot, &iv.eb.s_halo));
    DWF_TRY(h->ws->get("ms_yh", per_site * H.He_tot, &iv.eb.y_halo));
  }
  }
  double *dsc, *blk;
  DWF_TRY(h->ws->get("ms_scal", S_NSLOT * sizeof(double), (void**)&dsc));
  DWF_TRY(h->ws->get("ms_blk", 5 * (size_t)gb.nblocks * sizeof(double), (void**)&blk));
  DWF_CUDA(cudaMemsetAsync(dsc, 0, S_NSLOT * sizeof(double), h->stream));

  DWF_TRY(pack_even(h, layL, b_c128, b64, P64, 1.0));
  DWF_TRY(vop(E64, VOP_ZERO, nullptr, x64));
  double bb, rr64, rrm;
  DWF_TRY(true_residual(E64, b64, nullptr, r64, t1, t2, t3, dsc, &bb));
  if (!(bb > 0.0) || !std::isfinite(bb)) {
    if (bb == 0.0) {
      DWF_TRY(unpack_even(h, layL, x64, P64, x_c128, 1.0));
      DWF_CUDA(cudaStreamSynchronize(h->stream));
      return DWF_OK;
    }
    return set_error(DWF_ERR_BREAKDOWN, "source norm is not finite");
  }
  rr64 = bb;
  const double tol2 = tol * tol * bb;
  const double delta = (middle == P64) ? 0.0 : ru_delta();
  const int nbk = gb.nblocks;

  DWF_TRY(cast(Em, P64, r64, rm, 1.0, nullptr, 0, nullptr, Em.red(FIN_STORE, dsc + S_RR)));
  DWF_TRY(vop(Em, VOP_ZERO, nullptr, xm));
  DWF_TRY(vop(Em, VOP_ZERO, nullptr, pm));
  if (flex) DWF_TRY(vop(Em, VOP_ZERO, nullptr, rold));
  ZSrc zs;
  PcGraph pg;
  DWF_TRY(precondition(Em, Ei, rm, zm, iv, dsc, blk, nbk, l, flex, rold, zs, &pg));
  // x += alpha p of an outer iteration is deferred into the next update of p (one pass over
  // x and p instead of two) unless a reliable update needs x first
  bool x_pending = false;
  auto flush_x = [&]() -> dwf_status {
    if (!x_pending) return DWF_OK;
    x_pending = false;
    VecArgs va{};
    va.x = xm;
    va.p = pm;
    va.Vp = g.Vp;
    va.Vhb = g.Vhb;
    va.Vhb_pad = g.Vhb_pad;
    va.alpha = dsc + S_ALPHA;
    va.seg_cps = Em.seg_cps;
    va.do_x = 1;
    return vec(Em, va);
  };
  auto update_p = [&]() -> dwf_status {
    VecArgs va{};
    if (x_pending) {   // x += alpha p with the old p, then p = z + beta p
      va.x = xm;
      va.alpha = dsc + S_ALPHA;
      va.do_x = 1;
      x_pending = false;
    }
    va.p = pm;
    va.r = zm;
    va.z_src = zs.src;
    va.z_prec = zs.prec;
    va.z_map = zs.map;
    va.z_vp = zs.vp;
    va.z_num = zs.num;
    va.z_den = zs.den;
    va.u = um;
    va.Vp = g.Vp;
    va.Vhb = g.Vhb;
    va.Vhb_pad = g.Vhb_pad;
    va.beta = dsc + S_BETA;
    va.seg_cps = Em.seg_cps;
    va.do_p = 1;
    va.do_u = Em.trivial() ? 0 : 1;
    va.db = h->b;
    va.dc = h->c;
    va.mf = h->mf;
    return vec(Em, va, zs.bytes);
  };
  DWF_TRY(update_p());
  double anchor = rr64;
  int k = 0, inner_total = l;
  dwf_status status = DWF_ERR_NOT_CONVERGED;
  std::vector<double> hist;
  set_error(DWF_ERR_NOT_CONVERGED, "maximum number of iterations reached");
  while (k < maxit) {
    RedArgs ra = Em.red(FIN_ALPHA, dsc + S_PAP);
    ra.rho = dsc + S_RHO;
    ra.alpha = dsc + S_ALPHA;
    DWF_TRY(Em.mpc(pm, um, tm, ym, EPI_NORM, ra, nullptr, true));
    if (flex) DWF_TRY(vop(Em, VOP_COPY, rm, rold));
    DWF_TRY(Em.mpcdag(ym, sm, nullptr, EPI_CG_R, rm, dsc + S_ALPHA,
                      Em.red(FIN_STORE, dsc + S_RR), nullptr));
    x_pending = true;
    k++;
    DWF_TRY(read_doubles(h, dsc + S_RR, 1, &rrm));
    hist.push_back(std::sqrt(rrm / bb));
    if (!std::isfinite(rrm)) {
      status = set_error(DWF_ERR_BREAKDOWN, "residual is not finite");
      break;
    }
    if (rrm <= tol2 || rrm <= delta * delta * anchor) {
      DWF_TRY(flush_x());
      DWF_TRY(vop(E64, VOP_ADD_CAST, xm, x64, RedArgs{}, 1.0, nullptr, middle));
      DWF_TRY(true_residual(E64, b64, x64, r64, t1, t2, t3, dsc, &rr64));
      if (stats) stats->reliable_updates++;
      if (rr64 <= tol2) {
        status = DWF_OK;
        break;
      }
      DWF_TRY(cast(Em, P64, r64, rm, 1.0, nullptr, 0, nullptr, Em.red(FIN_STORE, dsc + S_RR)));
      DWF_TRY(vop(Em, VOP_ZERO, nullptr, xm));
      anchor = rr64;
    }
    DWF_TRY(precondition(Em, Ei, rm, zm, iv, dsc, blk, nbk, l, flex, rold, zs, &pg));
    inner_total += l;
    DWF_TRY(update_p());
  }
  if (status == DWF_ERR_NOT_CONVERGED) {
    // fold the current middle iterate into the FP64 solution
    DWF_TRY(flush_x());
    DWF_TRY(vop(E64, VOP_ADD_CAST, xm, x64, RedArgs{}, 1.0, nullptr, middle));
    DWF_TRY(true_residual(E64, b64, x64, r64, t1, t2, t3, dsc, &rr64));
  }
  DWF_TRY(unpack_even(h, layL, x64, P64, x_c128, 1.0));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  if (stats) {
    stats->iterations = k;
    stats->inner_iterations = inner_total;
    stats->operator_applications = k + stats->reliable_updates;
    stats->true_residual = std::sqrt(rr64 / bb);
    if (stats->history && stats->history_capacity > 0) {
      const int n = std::min((int)hist.size(), stats->history_capacity);
      for (int i = 0; i < n; i++) stats->history[i] = hist[i];
      stats->history_len = n;
    }
    stats->seconds = timer.seconds();
  }
  return status;
}

}  // namespace dwf

extern "C" dwf_status dwf_mspcg(dwf_t h, const int block[4], int inner_iters, dwf_prec inner,
                                dwf_prec middle, dwf_local_op local_op, int flexible,
                                const void* phi, void* x, double tol, int maxit,
                                dwf_stats* stats) {
  if (!h || !block || !phi || !x) return set_error(DWF_ERR_ARG, "null argument");
  if (inner_iters < 1) return set_error(DWF_ERR_ARG, "inner_iters must be >= 1");
  if (!(tol > 0.0) || maxit < 0) return set_error(DWF_ERR_ARG, "bad tolerance or maxit");
  if ((int)inner < 0 || (int)inner > 3) return set_error(DWF_ERR_ARG, "bad inner precision");
  if (middle != DWF_F32 && middle != DWF_F64)
    return set_error(DWF_ERR_ARG, "middle precision must be DWF_F32 or DWF_F64");
  if (local_op != DWF_LOCAL_DROP && local_op != DWF_LOCAL_EXACT)
    return set_error(DWF_ERR_ARG, "unknown local_op");
  Layout* lay;
  DWF_TRY(get_layout(h, block, &lay));
  Layout* layL;
  DWF_TRY(get_layout(h, h->dims, &layL));
  const size_t ub = (size_t)h->Ls * (lay->g.V / 2) * 12 * 16;
  void *db, *dx;
  DWF_TRY(stage_buffer(h, "io_phi", phi, ub, true, &db));
  DWF_TRY(stage_buffer(h, "io_x", x, ub, false, &dx));
  dwf_status st = run_mspcg(h, lay, layL, inner_iters, (int)inner, (int)middle, flexible != 0,
                            local_op == DWF_LOCAL_EXACT, db, dx, tol, maxit, stats);
  if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
  dwf_status st2 = finish_output(h, x, dx, ub);
  return st2 != DWF_OK ? st2 : st;
}

// ---------------------------------------------------------------------------------------
// Stationary block iterations: the multisplitting iteration (Sec. 2.1, Eq. 2) and the
// multiplicative Schwarz sweeps over 2- and 16-colour checkerboards of blocks.
// ---------------------------------------------------------------------------------------
namespace dwf {

static dwf_status run_ms(dwf_ctx* h, Layout* lay, Layout* layL, int l, int inner, bool exact,
                         int ncol, const void* b_c128, void* x_c128, double tol, int maxit,
                         dwf_stats* stats) {
  Timer timer;
  stats_init(stats);
  const Geom& g = layL->g;
  OpEngine E64;
  DWF_TRY(E64.init(h, layL, P64, false));
  DWF_TRY(ensure_reduction(h, g.Vp / 32 * 2 + 64, 64));
  SimdLocal* S;
  DWF_TRY(ensure_simd(h, lay, exact, &S));
  const size_t f64 = field_bytes(g, P64);
  void *b64, *x64, *r64, *z64, *t1, *t2, *t3;
  DWF_TRY(h->ws->get("ms_b64", f64, &b64));
  DWF_TRY(h->ws->get("ms_x64", f64, &x64));
  DWF_TRY(h->ws->get("ms_r64", f64, &r64));
  DWF_TRY(h->ws->get("ms_zm", f64, &z64));
  DWF_TRY(h->ws->get("ms_t1", f64, &t1));
  DWF_TRY(h->ws->get("ms_t2", f64, &t2));
  DWF_TRY(h->ws->get("ms_t3", f64, &t3));
  const size_t per = (size_t)h->Ls * 24 * real_bytes(inner);
  SimdFields F{};
  DWF_TRY(h->ws->get("ms_xi", per * S->sB, &F.x));
  DWF_TRY(h->ws->get("ms_pi", per * S->sB, &F.p));
  DWF_TRY(h->ws->get("ms_ui", per * S->sB, &F.u));
  DWF_TRY(h->ws->get("ms_ri", per * S->sB, &F.r));
  DWF_TRY(h->ws->get("ms_ti", per * S->sO, &F.t));
  DWF_TRY(h->ws->get("ms_yi", per * S->sE, &F.y));
  double* dsc;
  DWF_TRY(h->ws->get("ms_scal", S_NSLOT * sizeof(double), (void**)&dsc));
  DWF_TRY(pack_even(h, layL, b_c128, b64, P64, 1.0));
  DWF_TRY(vop(E64, VOP_ZERO, nullptr, x64));
  double bb, rr;
  DWF_TRY(true_residual(E64, b64, nullptr, r64, t1, t2, t3, dsc, &bb));
  if (!(bb > 0.0) || !std::isfinite(bb)) {
    if (bb == 0.0) {
      DWF_TRY(unpack_even(h, layL, x64, P64, x_c128, 1.0));
      DWF_CUDA(cudaStreamSynchronize(h->stream));
      return DWF_OK;
    }
    return set_error(DWF_ERR_BREAKDOWN, "source norm is not finite");
  }
  rr = bb;
  const bool scaled = (inner == P16 || inner == PB16);
  const double nreal = 24.0 * h->Ls * (double)(g.V / 2);
  std::vector<double> hist;
  int k = 0, applications = 0;
  dwf_status status = set_error(DWF_ERR_NOT_CONVERGED, "maximum number of sweeps reached");
  while (k < maxit && rr > tol * tol * bb) {
    for (int c = 0; c < ncol; c++) {
      // z = local solves of the blocks of colour c on the current residual (|r|^2 in S_TMP),
      // x += z, r = b - A x
      DWF_TRY(simd_local_solve(h, S, inner, l, r64, P64, g.Vp, scaled ? nreal : 1.0,
                               scaled ? dsc + S_TMP : nullptr, F, ncol, c));
      DWF_TRY(cast(E64, inner, F.x, z64, scaled ? nreal : 1.0, scaled ? dsc + S_TMP : nullptr,
                   1, nullptr, RedArgs{}, nullptr, S->inv, S->sB));
      DWF_TRY(vop(E64, VOP_AXPY, z64, x64, RedArgs{}, 1.0));
      DWF_TRY(true_residual(E64, b64, x64, r64, t1, t2, t3, dsc, &rr));
      applications++;
    }
    k++;
    hist.push_back(std::sqrt(rr / bb));
    if (!std::isfinite(rr)) {
      status = set_error(DWF_ERR_BREAKDOWN, "residual is not finite");
      break;
    }
  }
  if (rr <= tol * tol * bb) status = DWF_OK;
  DWF_TRY(check_device_error(h));
  DWF_TRY(unpack_even(h, layL, x64, P64, x_c128, 1.0));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  if (stats) {
    stats->iterations = k;
    stats->inner_iterations = k * ncol * l;
    stats->operator_applications = applications;
    stats->true_residual = std::sqrt(rr / bb);
    if (stats->history && stats->history_capacity > 0) {
      const int n = std::min((int)hist.size(), stats->history_capacity);
      for (int i = 0; i < n; i++) stats->history[i] = hist[i];
      stats->history_len = n;
    }
    stats->seconds = timer.seconds();
  }
  return status;
}

}  // namespace dwf

extern "C" dwf_status dwf_ms_solve(dwf_t h, const int block[4], int inner_iters,
                                   dwf_prec inner, dwf_local_op local_op, int colours,
                                   const void* phi, void* x, double tol, int maxit,
                                   dwf_stats* stats) {
  if (!h || !block || !phi || !x) return set_error(DWF_ERR_ARG, "null argument");
  if (inner_iters < 1) return set_error(DWF_ERR_ARG, "inner_iters must be >= 1");
  if (!(tol >= 0.0) || maxit < 0) return set_error(DWF_ERR_ARG, "bad tolerance or maxit");
  if ((int)inner < 0 || (int)inner > 3) return set_error(DWF_ERR_ARG, "bad inner precision");
  if (local_op != DWF_LOCAL_DROP && local_op != DWF_LOCAL_EXACT)
    return set_error(DWF_ERR_ARG, "unknown local_op");
  if (colours != 1 && colours != 2 && colours != 16)
    return set_error(DWF_ERR_ARG, "colours must be 1, 2 or 16");
  Layout* lay;
  DWF_TRY(get_layout(h, block, &lay));
  if (colours > 1)
    for (int m = 0; m < 4; m++)
      if (lay->g.nb[m] > 1 && lay->g.nb[m] % 2 != 0)
        return set_error(DWF_ERR_ARG, "a checkerboard of blocks needs an even number of "
                                      "blocks (or one) in every direction");
  Layout* layL;
  DWF_TRY(get_layout(h, h->dims, &layL));
  const size_t ub = (size_t)h->Ls * (lay->g.V / 2) * 12 * 16;
  void *db, *dx;
  DWF_TRY(stage_buffer(h, "io_phi", phi, ub, true, &db));
  DWF_TRY(stage_buffer(h, "io_x", x, ub, false, &dx));
  dwf_status st = run_ms(h, lay, layL, inner_iters, (int)inner, local_op == DWF_LOCAL_EXACT,
                         colours, db, dx, tol, maxit, stats);
  if (st != DWF_OK && st != DWF_ERR_NOT_CONVERGED) return st;
  dwf_status st2 = finish_output(h, x, dx, ub);
  return st2 != DWF_OK ? st2 : st;
}
