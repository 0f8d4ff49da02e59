// Operator engine: the stage launches that make up Mpc, Mpc^dag, D and D^dag on one site
// ordering and one storage precision, plus the handle's device workspace.
#pragma once

#include <cstdio>
#include <string>
#include <unordered_map>

#include "dwf_internal.h"

namespace dwf {

struct Workspace {
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::unordered_map<std::string, Buf> bufs;
  ~Workspace() {
    for (auto& kv : bufs) cudaFree(kv.second.p);
  }
  // Device buffer of at least `bytes` under `name` (allocated once, kept for the handle).
  dwf_status get(const std::string& name, size_t bytes, void** out) {
    Buf& b = bufs[name];
    if (b.bytes < bytes) {
      cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
      if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DWF_ERR_NOMEM, "workspace allocation failed: " + name);
      }
      b.bytes = bytes;
    }
    *out = b.p;
    return DWF_OK;
  }
};

struct OpEngine {
  dwf_ctx* h = nullptr;
  Layout* lay = nullptr;
  int prec = P64;
  bool blocked = false;
  int seg_cps = 1;   // CTAs per scalar segment: whole grid, or one lattice block
  const void* links[2] = {nullptr, nullptr};

  dwf_status init(dwf_ctx* hh, Layout* l, int p, bool blk) {
    h = hh;
    lay = l;
    prec = p;
    blocked = blk;
    DWF_TRY(ensure_links(h, lay, prec));
    links[0] = lay->links[prec][0];
    links[1] = lay->links[prec][1];
    seg_cps = blk ? lay->g.Vhb_pad / 32 : (int)(lay->g.Vp / 32);
    return DWF_OK;
  }
  RedArgs red(int op, double* res) const { return make_red(h, seg_cps, op, res); }
  int cls() const { return prec == P64 ? 0 : 1; }
  // how a stage applies D+ M5op^-1 / M5op^-dag D+^dag (call after post_h is set)
  void set_struct(StageArgs& a) const {
    const Matrices& M = h->mats;
    if (!M.struct_ok || M.post_mode == 1) return;
    a.post_struct = (M.post_mode == 0 && a.post_h) ? 2 : 1;
    a.dp_b = h->b;
    a.dp_c = h->c;
    a.post_pre = trivial() ? h->b : 1.0;
  }
  // FP16 tensor-core operand of post matrix w (0: D+ M5op^-1, 1: M5op^-dag D+^dag, 2: D+^dag)
  const void* post_h(int w) const {
    return ((prec == P16 || prec == PB16) && h->mats.use_tc) ? h->mats.d_post_h[w] : nullptr;
  }
  bool trivial() const { return h->mats.dplus_trivial; }
  const Geom& g() const { return lay->g; }

  StageArgs base(int out_par) const {
    StageArgs a{};
    a.links = links[out_par];
    a.nbr = lay->nbr[out_par];
    a.Vp = lay->g.Vp;
    a.Vp_in = lay->g.Vp;
    a.Vp_halo = lay->g.Vp;
    a.Vp_link = lay->g.Vp;
    a.Vhb = lay->g.Vhb;
    a.Vhb_pad = lay->g.Vhb_pad;
    a.hop_scale = 1.0;
    a.mf = h->mf;
    a.l_alpha = h->mats.m5_alpha;
    a.l_beta = h->mats.m5_beta;
    a.seg_cps = seg_cps;
    a.err = h->dev_err;
    a.wait_ns = h->wait_ns;
    a.wait_probe = h->wait_probe;
    return a;
  }
  dwf_status launch(const StageArgs& a, bool dag) const {
    // algorithmic bytes: hop input, output, optional local input and residual read, once per
    // site and slice; the 8 links of each output site once
    const double R = (double)real_bytes(prec);
    const double sites = (double)(a.Vp / a.Vhb_pad) * a.Vhb;
    const double per_ss = 24.0 * R * (2.0 + (a.local_mode != LOC_NONE) + (a.epi == EPI_CG_R) -
                                      (a.epi == EPI_NORM_ONLY));
    const double bytes = sites * h->Ls * per_ss + sites * 8 * 18 * R;
    const char* kind = a.Vp != lay->g.Vp ? "halo" : (blocked ? "blocked" : "full");
    char name[48];
    // _m5: dense D+ M5op^-1 / M5op^-dag D+^dag post; _dp: sparse D+^dag post
    snprintf(name, sizeof(name), "hop_%s_%s%s", prec_name(prec), kind,
             a.post ? (a.post_sparse ? "_dp" : "_m5") : "");
    ProfScope ps(&h->prof, h->stream, name, bytes, 1320.0 * sites * h->Ls);
    DWF_CUDA(launch_stage_prec(prec, a, h->Ls, dag, blocked, h->stream));
    return DWF_OK;
  }

  // u = D+ x (Moebius pre-op); also used with do_x/do_p off.
  dwf_status dplus(const void* x, void* u, const int* stop) const {
    VecArgs v{};
    v.p = const_cast<void*>(x);
    v.u = u;
    v.Vp = lay->g.Vp;
    v.Vhb = lay->g.Vhb;
    v.Vhb_pad = lay->g.Vhb_pad;
    v.do_u = 1;
    v.seg_cps = seg_cps;
    v.db = h->b;
    v.dc = h->c;
    v.mf = h->mf;
    v.stop = stop;
    ProfScope ps(&h->prof, h->stream, "dplus", 2.0 * field_bytes(lay->g, prec), 0.0);
    DWF_CUDA(launch_vec(prec, v, h->Ls, h->stream));
    return DWF_OK;
  }

  // y = Mpc x.  u: even temporary (D+ x, unused when D+ = b), t: odd temporary.
  dwf_status mpc(const void* x, void* u, void* t, void* y, int epi, const RedArgs& red,
                 const int* stop, bool u_ready = false) const {
    const void* xin = x;
    if (!trivial()) {
      if (!u_ready) DWF_TRY(dplus(x, u, stop));
      xin = u;
    }
    StageArgs a = base(1);
    a.in = xin;
    a.out = t;
    a.post = h->mats.d_dpm5i[cls()];
    a.post_h = post_h(0);
    set_struct(a);
    a.epi = EPI_STORE;
    a.stop = stop;
    DWF_TRY(launch(a, false));
    StageArgs b = base(0);
    b.in = t;
    b.out = y;
    b.in2 = x;
    b.local_mode = LOC_M5;
    b.hop_scale = -0.25;
    b.epi = epi;
    b.red = red;
    b.stop = stop;
    return launch(b, false);
  }

  // z = Mpc^dag y (epi EPI_CG_R: r -= alpha z instead of storing z).  s: odd temporary.
  dwf_status mpcdag(const void* y, void* sb, void* z, int epi, void* r, const double* alpha,
                    const RedArgs& red, const int* stop) const {
    StageArgs a = base(1);
    a.in = y;
    a.out = sb;
    a.post = h->mats.d_m5idpt[cls()];
    a.post_h = post_h(1);
    set_struct(a);
    a.epi = EPI_STORE;
    a.stop = stop;
    DWF_TRY(launch(a, true));
    StageArgs b = base(0);
    b.in = sb;
    b.out = z;
    b.in2 = y;
    b.local_mode = LOC_M5DAG;
    if (trivial()) {
      b.hop_scale = -0.25 * h->b;
    } else {
      b.hop_scale = -0.25;
      b.post = h->mats.d_dpt[cls()];
      b.post_sparse = 1;
      b.dp_b = h->b;
      b.dp_c = h->c;
    }
    b.epi = epi;
    b.r = r;
    b.alpha = alpha;
    b.red = red;
    b.stop = stop;
    return launch(b, true);
  }

  // ---- exact block operator A_s = P_s Mpc^dag Mpc P_s, every block at once ----
  // y = Mpc P_s p lives on the block and its even halo; the odd intermediates on the block and
  // its odd halo.  Each block owns its halo arrays, so blocks never mix.
  struct ExactBufs {
    void *t_int, *t_halo, *y_int, *y_halo, *s_int, *s_halo;
  };
  StageArgs halo_base(int out_par, bool odd_halo) const {
    StageArgs a = base(out_par);
    const Halo& H = *lay->halo;
    a.nbr = odd_halo ? H.nbr_ho : H.nbr_he;
    a.Vp = odd_halo ? H.Ho_tot : H.He_tot;
    a.Vhb = odd_halo ? H.Ho_b : H.He_b;
    a.Vhb_pad = odd_halo ? H.Ho_pad : H.He_pad;
    a.seg_cps = a.Vhb_pad / 32;
    a.links = odd_halo ? H.links_ho[prec] : H.links_he[prec];
    a.Vp_link = a.Vp;
    return a;
  }

  // y = Mpc P_s p (u = D+ p unless D+ = b); per block: pap_int = ||y||^2 on the block, then
  // alpha = rho / (||y||^2 on the block + on the halo).
  // store_y = false: only the norms are needed (no A^dag stage follows)
  dwf_status exact_mpc(const void* p, const void* u, const ExactBufs& B, double* pap_int,
                       double* rho, double* alpha, const int* stop, bool store_y = true) const {
    const Halo& H = *lay->halo;
    const void* xin = trivial() ? p : u;
    const void* X = h->mats.d_dpm5i[cls()];
    StageArgs a = base(1);
    a.nbr = H.nbr_bo;
    a.in = xin;
    a.skip_halo = 1;
    a.post = X;
    a.post_h = post_h(0);
    set_struct(a);
    a.out = B.t_int;
    a.stop = stop;
    DWF_TRY(launch(a, false));
    StageArgs b = halo_base(1, true);
    b.in = xin;
    b.skip_halo = 1;
    b.post = X;
    b.post_h = post_h(0);
    set_struct(b);
    b.out = B.t_halo;
    b.stop = stop;
    DWF_TRY(launch(b, false));
    StageArgs c = base(0);
    c.nbr = H.nbr_be;
    c.in = B.t_int;
    c.in_halo = B.t_halo;
    c.Vp_halo = H.Ho_tot;
    c.in2 = p;
    c.local_mode = LOC_M5;
    c.hop_scale = -0.25;
    c.out = B.y_int;
    c.epi = store_y ? EPI_NORM : EPI_NORM_ONLY;
    c.red = red(FIN_STORE, pap_int);
    c.stop = stop;
    DWF_TRY(launch(c, false));
    StageArgs d = halo_base(0, false);
    d.in = B.t_int;
    d.in_halo = B.t_halo;
    d.Vp_halo = H.Ho_tot;
    d.hop_scale = -0.25;
    d.out = B.y_halo;
    d.epi = store_y ? EPI_NORM : EPI_NORM_ONLY;
    d.red = make_red(h, H.He_pad / 32, FIN_ALPHA2, nullptr);
    d.red.rho = rho;
    d.red.alpha = alpha;
    d.red.extra = pap_int;
    d.stop = stop;
    return launch(d, false);
  }

  // r -= alpha P_s Mpc^dag y  with y from exact_mpc.
  dwf_status exact_mpcdag_cg(const ExactBufs& B, void* r, const double* alpha,
                             const RedArgs& rb, const int* stop) const {
    const Halo& H = *lay->halo;
    const void* Xd = h->mats.d_m5idpt[cls()];
    StageArgs a = base(1);
    a.nbr = H.nbr_bo;
    a.in = B.y_int;
    a.in_halo = B.y_halo;
    a.Vp_halo = H.He_tot;
    a.post = Xd;
    a.post_h = post_h(1);
    set_struct(a);
    a.out = B.s_int;
    a.stop = stop;
    DWF_TRY(launch(a, true));
    StageArgs b = halo_base(1, true);
    b.in = B.y_int;
    b.in_halo = B.y_halo;
    b.Vp_halo = H.He_tot;
    b.post = Xd;
    b.post_h = post_h(1);
    set_struct(b);
    b.out = B.s_halo;
    b.stop = stop;
    DWF_TRY(launch(b, true));
    StageArgs c = base(0);
    c.nbr = H.nbr_be;
    c.in = B.s_int;
    c.in_halo = B.s_halo;
    c.Vp_halo = H.Ho_tot;
    c.in2 = B.y_int;
    c.local_mode = LOC_M5DAG;
    if (trivial()) {
      c.hop_scale = -0.25 * h->b;
    } else {
      c.hop_scale = -0.25;
      c.post = h->mats.d_dpt[cls()];
      c.post_sparse = 1;
      c.dp_b = h->b;
      c.dp_c = h->c;
    }
    c.epi = EPI_CG_R;
    c.r = r;
    c.alpha = alpha;
    c.red = rb;
    c.stop = stop;
    return launch(c, true);
  }

  // Full operator on (even, odd) halves: out_p = M5op x_p - 1/2 Dh_{p,1-p} D+ x_{1-p}
  // (dag: out_p = M5op^dag x_p - 1/2 D+^dag Dh^dag_{p,1-p} x_{1-p}).
  dwf_status full(const void* xe, const void* xo, void* ue, void* uo, void* oe, void* oo,
                  bool dag) const {
    const void* x[2] = {xe, xo};
    void* u[2] = {ue, uo};
    void* o[2] = {oe, oo};
    if (!dag && !trivial()) {
      DWF_TRY(dplus(xe, ue, nullptr));
      DWF_TRY(dplus(xo, uo, nullptr));
    }
    for (int p = 0; p < 2; p++) {
      StageArgs a = base(p);
      a.out = o[p];
      a.in2 = x[p];
      a.epi = EPI_STORE;
      if (!dag) {
        a.in = trivial() ? x[1 - p] : u[1 - p];
        a.local_mode = LOC_M5;
        a.hop_scale = trivial() ? -0.5 * h->b : -0.5;
      } else {
        a.in = x[1 - p];
        a.local_mode = LOC_M5DAG;
        if (trivial()) {
          a.hop_scale = -0.5 * h->b;
        } else {
          a.hop_scale = -0.5;
          a.post = h->mats.d_dpt[cls()];
          a.post_sparse = 1;
          a.dp_b = h->b;
          a.dp_c = h->c;
        }
      }
      DWF_TRY(launch(a, dag));
    }
    return DWF_OK;
  }
};

}  // namespace dwf
