// Batched solver: many independent problems A_i x_i = phi_i, each with its own lattice, Ls,
// masses and links, solved together.
//
// Problems with the same Ls share one concatenated site space (each problem padded to whole
// 32-site tiles); every problem is one reduction/scalar segment with its own fifth-dimension
// matrices, M5op coefficients, stop flag and CG scalars.  A chunk of 16 FP32 CG steps of every
// problem of a group is either one persistent, cooperative launch (batch_steps.cu: five
// phases per step over all tiles, grid barriers with bounded waits) or five launches per step
// (stages A, B, A^dag, B^dag on persistent grids, then the update); which one, the grid size
// and the link staging are picked per group by timing the first chunks (and kept for later
// calls on the same problem mix), and the chosen launches of all groups are then captured
// once in a CUDA graph and replayed.  FP32 CG with
// FP64 reliable updates per problem (the true residual is recomputed in FP64 when a problem's
// FP32 residual has dropped by delta = 0.1, or at convergence), between replays.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace dwf {

namespace {

struct Prob {
  int dims[4];
  int Ls;
  double M5, mf, b, c;
  long V, Vh, Vp;       // sites, sites of one parity, padded
  long first_tile, ntiles;
  long off_links;       // offset (complex elements) of its links in the staged copy
};

struct Group {
  int Ls = 0;
  std::vector<int> ids;        // problem indices
  long ntiles = 0, Vp = 0;
  int nseg = 0;
  uint32_t* nbr[2] = {};
  int* lex[2] = {};
  int* tile_seg = nullptr;
  BatchSeg* segp[2] = {};      // [0] FP64 matrices, [1] FP32 matrices
  void* mats[2] = {};
  void* links[2][2] = {};      // [0 f64, 1 f32][parity]
  const double2** srcs = nullptr;   // per segment caller source / solution pointers
  double2** dsts = nullptr;
  void* f64[6] = {};           // b, x, r, t1, t2, t3
  void* f32[7] = {};           // x, p, r, u, t, y, s
  double* sc = nullptr;        // [8][nseg]: rho, alpha, beta, pap, stop2, rr64, bb, tmp
  int* fl = nullptr;           // [4][nseg]: conv, stop, iter, skip (RU selection)
  unsigned* counter = nullptr; // [nseg]
  double* partial = nullptr;   // [ntiles]
  int grid = 0;                // autotuned persistent grid of the stage launches
  int sgrid = 0, sgather = -1;  // persistent CG-step launch: grid, link staging (tuned;
                                // gather -1: one launch per stage instead)
  unsigned* bar = nullptr;     // barrier counter of the persistent launch
  int* err = nullptr;          // set when a bounded device wait gives up
  int post_struct = 1;         // every problem has |beta/alpha| < 1: post by recurrences
  std::vector<void*> owned;
  ~Group() {
    for (void* p : owned) cudaFree(p);
  }
  template <typename T>
  dwf_status alloc(T** p, size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(DWF_ERR_NOMEM, "batched solver: device allocation failed");
    }
    owned.push_back(q);
    *p = static_cast<T*>(q);
    return DWF_OK;
  }
};

enum { SC_RHO = 0, SC_ALPHA, SC_BETA, SC_PAP, SC_STOP2, SC_RR64, SC_BB, SC_TMP, SC_N };
enum { FL_CONV = 0, FL_STOP, FL_ITER, FL_SKIP, FL_N };

long plain_index(const int d[4], const int c[4]) {
  return c[0] / 2 + (long)(d[0] / 2) * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3]));
}

// ---- kernels specific to the batch (caller layouts of several problems) ----
template <int P>
__global__ void batch_pack_links_kernel(const double2* __restrict__ U, void* out,
                                        const uint32_t* __restrict__ nbr,
                                        const int* __restrict__ lexp, const int* __restrict__ lexq,
                                        const int* __restrict__ tile_seg, const long* link_off,
                                        long Vp) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (idx >= Vp) return;
  const int mu = d >> 1, back = d & 1;
  const int lx = lexp[idx];
  double re[9], im[9];
  if (lx < 0) {
    for (int k = 0; k < 9; k++) re[k] = im[k] = 0.0;
  } else {
    const double2* Uq = U + link_off[tile_seg[idx >> 5]];
    if (!back) {
      const double2* u = Uq + ((long)lx * 4 + mu) * 9;
      for (int k = 0; k < 9; k++) {
        re[k] = u[k].x;
        im[k] = u[k].y;
      }
    } else {
      const int nl = lexq[nbr[(long)d * Vp + idx] & NBR_IDX];
      const double2* u = Uq + ((long)nl * 4 + mu) * 9;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          re[a * 3 + b] = u[b * 3 + a].x;
          im[a * 3 + b] = -u[b * 3 + a].y;
        }
    }
  }
  // same 16-byte chunk layout as the single-problem links
  constexpr int NCHL = Prec<P>::NCHL;
  uint4* o = reinterpret_cast<uint4*>(out) + (long)d * NCHL * Vp + idx;
  if constexpr (P == P64) {
    for (int k = 0; k < 9; k++) *reinterpret_cast<double2*>(o + k * Vp) = make_double2(re[k], im[k]);
  } else {
    for (int k = 0; k < 5; k++) {
      const int a = 2 * k, b = 2 * k + 1;
      *reinterpret_cast<float4*>(o + k * Vp) = make_float4(
          (float)re[a], (float)im[a], b < 9 ? (float)re[b] : 0.f, b < 9 ? (float)im[b] : 0.f);
    }
  }
}

// Caller even-half c128 of problem q <-> the group's concatenated FP64 field.
__global__ void batch_move_kernel(const double2* const* srcs, double2* const* dsts, double2* f,
                                  const int* __restrict__ tile_seg, const BatchSeg* segp,
                                  const int* skip, long Vp, int to_field) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (idx >= Vp) return;
  const int q = tile_seg[idx >> 5];
  if (skip && skip[q]) return;
  const BatchSeg& S = segp[q];
  const long j = idx - (long)S.first_tile * 32;
  // FP64 field chunk layout: [s][12][Vp] of double2
  double2* fp = f + ((long)s * 12) * Vp + idx;
  if (j >= S.Vh) {
    if (to_field)
      for (int k = 0; k < 12; k++) fp[k * Vp] = make_double2(0.0, 0.0);
    return;
  }
  if (to_field) {
    const double2* src = srcs[q] + ((long)s * S.Vh + j) * 12;
    for (int k = 0; k < 12; k++) fp[k * Vp] = src[k];
  } else {
    double2* dst = dsts[q] + ((long)s * S.Vh + j) * 12;
    for (int k = 0; k < 12; k++) dst[k] = fp[k * Vp];
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------------------
namespace {

struct Batch {
  std::vector<Prob> probs;
  std::vector<std::unique_ptr<Group>> groups;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  double* staged_links = nullptr;
  unsigned long long wait_ns = 0;   // bounded device waits (DWF_WAIT_LIMIT_US; 0: default)
  std::vector<void*> owned;
  ~Batch() {
    if (st) cudaStreamSynchronize(st);
    groups.clear();
    for (void* p : owned) cudaFree(p);
    if (own_stream) cudaStreamDestroy(st);
  }
};

StageArgs gbase(const Group& G, int prec, int out_par, const int* stop) {
  StageArgs a{};
  a.links = G.links[prec == P64 ? 0 : 1][out_par];
  a.nbr = G.nbr[out_par];
  a.Vp = a.Vp_in = a.Vp_halo = a.Vp_link = G.Vp;
  a.Vhb = (int)G.Vp;
  a.Vhb_pad = (int)G.Vp;
  a.seg_cps = (int)G.ntiles;
  a.hop_scale = 1.0;
  a.epi = EPI_STORE;
  a.stop = stop;
  a.tile_seg = G.tile_seg;
  a.segp = G.segp[prec == P64 ? 0 : 1];
  a.ntiles = G.ntiles;
  a.grid = G.grid;
  return a;
}

RedArgs gred(const Group& G, int op) {
  RedArgs r{};
  r.partial = G.partial;
  r.counter = G.counter;
  r.cps = (int)G.ntiles;
  r.op = op;
  return r;
}

// y = Mpc x (D+ x in u), with optional ||y||^2 -> alpha per problem.
dwf_status g_mpc(const Group& G, int prec, const void* x, void* u, void* t, void* y, bool alpha,
                 const int* stop, cudaStream_t st) {
  VecArgs v{};
  v.p = const_cast<void*>(x);
  v.u = u;
  v.Vp = G.Vp;
  v.Vhb = (int)G.Vp;
  v.Vhb_pad = (int)G.Vp;
  v.seg_cps = (int)G.ntiles;
  v.do_u = 1;
  v.stop = stop;
  v.tile_seg = G.tile_seg;
  v.segp = G.segp[prec == P64 ? 0 : 1];
  DWF_CUDA(launch_vec(prec, v, G.Ls, st));
  StageArgs a = gbase(G, prec, 1, stop);
  a.in = u;
  a.out = t;
  a.post = G.mats[0];   // non-null marks a post stage; the problem's matrix comes from segp
  a.post_which = 0;
  a.post_struct = G.post_struct;
  a.post_pre = 1.0;
  DWF_CUDA(launch_stage_prec(prec, a, G.Ls, false, false, st));
  StageArgs b = gbase(G, prec, 0, stop);
  b.in = t;
  b.out = y;
  b.in2 = x;
  b.local_mode = LOC_M5;
  b.hop_scale = -0.25;
  if (alpha) {
    b.epi = EPI_NORM;
    b.red = gred(G, FIN_ALPHA);
    b.red.res = G.sc + SC_PAP * G.nseg;
    b.red.rho = G.sc + SC_RHO * G.nseg;
    b.red.alpha = G.sc + SC_ALPHA * G.nseg;
  }
  DWF_CUDA(launch_stage_prec(prec, b, G.Ls, false, false, st));
  return DWF_OK;
}

// z = Mpc^dag y, or (cg) r -= alpha Mpc^dag y with ||r||^2 -> beta and convergence flags.
dwf_status g_mpcdag(const Group& G, int prec, const void* y, void* sb, void* z, void* r, bool cg,
                    const int* stop, cudaStream_t st) {
  StageArgs a = gbase(G, prec, 1, stop);
  a.in = y;
  a.out = sb;
  a.post = G.mats[0];
  a.post_which = 1;
  a.post_struct = G.post_struct;
  a.post_pre = 1.0;
  DWF_CUDA(launch_stage_prec(prec, a, G.Ls, true, false, st));
  StageArgs b = gbase(G, prec, 0, stop);
  b.in = sb;
  b.out = z;
  b.in2 = y;
  b.local_mode = LOC_M5DAG;
  b.hop_scale = -0.25;
  b.post = G.mats[0];
  b.post_which = 2;
  b.post_sparse = 1;   // D+^dag of each problem, from its segment's db, dc
  if (cg) {
    b.epi = EPI_CG_R;
    b.r = r;
    b.alpha = G.sc + SC_ALPHA * G.nseg;
    b.red = gred(G, FIN_BETA);
    b.red.rho = G.sc + SC_RHO * G.nseg;
    b.red.beta = G.sc + SC_BETA * G.nseg;
    b.red.stop2 = G.sc + SC_STOP2 * G.nseg;
    b.red.conv = G.fl + FL_CONV * G.nseg;
  }
  DWF_CUDA(launch_stage_prec(prec, b, G.Ls, true, false, st));
  return DWF_OK;
}

dwf_status g_vop(const Group& G, int prec, int op, const void* x, void* y, const int* stop,
                 int red_op, double* res, cudaStream_t st, int prec_x = -1, double sa = 1.0) {
  VopArgs a{};
  a.op = op;
  a.x = x;
  a.y = y;
  a.Vp = G.Vp;
  a.Vhb = (int)G.Vp;
  a.Vhb_pad = (int)G.Vp;
  a.sa = sa;
  a.stop = stop;
  a.tile_seg = G.tile_seg;
  a.segp = G.segp[0];
  if (res) {
    a.red = gred(G, red_op);
    a.red.res = res;
  }
  DWF_CUDA(launch_vop(prec, prec_x < 0 ? prec : prec_x, a, G.Ls, st));
  return DWF_OK;
}

// One FP32 CG step of every active problem of the group.
dwf_status g_cg_step(const Group& G, cudaStream_t st) {
  const int* stop = G.fl + FL_STOP * G.nseg;
  void** v = const_cast<void**>(G.f32);   // x, p, r, u, t, y, s
  // u = D+ p is kept by the update kernel; stage A reads it directly
  StageArgs a = gbase(G, P32, 1, stop);
  a.in = v[3];
  a.out = v[4];
  a.post = G.mats[1];
  a.post_which = 0;
  a.post_struct = G.post_struct;
  a.post_pre = 1.0;
  DWF_CUDA(launch_stage_prec(P32, a, G.Ls, false, false, st));
  StageArgs b = gbase(G, P32, 0, stop);
  b.in = v[4];
  b.out = v[5];
  b.in2 = v[1];
  b.local_mode = LOC_M5;
  b.hop_scale = -0.25;
  b.epi = EPI_NORM;
  b.red = gred(G, FIN_ALPHA);
  b.red.res = G.sc + SC_PAP * G.nseg;
  b.red.rho = G.sc + SC_RHO * G.nseg;
  b.red.alpha = G.sc + SC_ALPHA * G.nseg;
  DWF_CUDA(launch_stage_prec(P32, b, G.Ls, false, false, st));
  DWF_TRY(g_mpcdag(G, P32, v[5], v[6], nullptr, v[2], true, stop, st));
  VecArgs u{};
  u.x = v[0];
  u.p = v[1];
  u.r = v[2];
  u.u = v[3];
  u.Vp = G.Vp;
  u.Vhb = (int)G.Vp;
  u.Vhb_pad = (int)G.Vp;
  u.alpha = G.sc + SC_ALPHA * G.nseg;
  u.beta = G.sc + SC_BETA * G.nseg;
  u.seg_cps = (int)G.ntiles;
  u.do_x = u.do_p = u.do_u = 1;
  u.stop = stop;
  u.red.counter = G.counter;
  u.stop_out = G.fl + FL_STOP * G.nseg;
  u.conv_in = G.fl + FL_CONV * G.nseg;
  u.iter = G.fl + FL_ITER * G.nseg;
  u.tile_seg = G.tile_seg;
  u.segp = G.segp[1];
  DWF_CUDA(launch_vec(P32, u, G.Ls, st));
  return DWF_OK;
}

// The launches of one CG step (as g_cg_step issues them) as arguments of the persistent
// kernel that runs `nsteps` steps in one launch.
void g_step_args(const Group& G, int nsteps, unsigned long long wait_ns, BatchStepArgs& b) {
  const int* stop = G.fl + FL_STOP * G.nseg;
  void** v = const_cast<void**>(G.f32);   // x, p, r, u, t, y, s
  b = BatchStepArgs{};
  StageArgs a = gbase(G, P32, 1, stop);
  a.in = v[3];
  a.out = v[4];
  a.post = G.mats[1];
  a.post_which = 0;
  a.post_struct = 1;
  a.post_pre = 1.0;
  StageArgs bb = gbase(G, P32, 0, stop);
  bb.in = v[4];
  bb.out = v[5];
  bb.in2 = v[1];
  bb.local_mode = LOC_M5;
  bb.hop_scale = -0.25;
  bb.epi = EPI_NORM;
  bb.red = gred(G, FIN_ALPHA);
  bb.red.res = G.sc + SC_PAP * G.nseg;
  bb.red.rho = G.sc + SC_RHO * G.nseg;
  bb.red.alpha = G.sc + SC_ALPHA * G.nseg;
  StageArgs ad = gbase(G, P32, 1, stop);
  ad.in = v[5];
  ad.out = v[6];
  ad.post = G.mats[1];
  ad.post_which = 1;
  ad.post_struct = 1;
  ad.post_pre = 1.0;
  StageArgs bd = gbase(G, P32, 0, stop);
  bd.in = v[6];
  bd.in2 = v[5];
  bd.local_mode = LOC_M5DAG;
  bd.hop_scale = -0.25;
  bd.post = G.mats[1];
  bd.post_which = 2;
  bd.post_sparse = 1;
  bd.epi = EPI_CG_R;
  bd.r = v[2];
  bd.alpha = G.sc + SC_ALPHA * G.nseg;
  bd.red = gred(G, FIN_BETA);
  bd.red.rho = G.sc + SC_RHO * G.nseg;
  bd.red.beta = G.sc + SC_BETA * G.nseg;
  bd.red.stop2 = G.sc + SC_STOP2 * G.nseg;
  bd.red.conv = G.fl + FL_CONV * G.nseg;
  StageArgs* st4[4] = {&a, &bb, &ad, &bd};
  for (StageArgs* x : st4) {
    x->err = G.err;
    x->wait_ns = wait_ns;
    x->grid = 0;
    finish_stage_args(*x, G.Ls);
  }
  b.A = a;
  b.B = bb;
  b.Ad = ad;
  b.Bd = bd;
  VecArgs& u = b.U;
  u.x = v[0];
  u.p = v[1];
  u.r = v[2];
  u.u = v[3];
  u.Vp = G.Vp;
  u.Vhb = (int)G.Vp;
  u.Vhb_pad = (int)G.Vp;
  u.alpha = G.sc + SC_ALPHA * G.nseg;
  u.beta = G.sc + SC_BETA * G.nseg;
  u.seg_cps = (int)G.ntiles;
  u.do_x = u.do_p = u.do_u = 1;
  u.stop = stop;
  u.red.counter = G.counter;
  u.stop_out = G.fl + FL_STOP * G.nseg;
  u.conv_in = G.fl + FL_CONV * G.nseg;
  u.iter = G.fl + FL_ITER * G.nseg;
  u.tile_seg = G.tile_seg;
  u.segp = G.segp[1];
  b.ntiles = G.ntiles;
  b.nsteps = nsteps;
  b.bar = G.bar;
  b.wait_ns = wait_ns;
  b.err = G.err;
}

// r64 = b - A64 x64 for the problems with skip == 0; ||r64||^2 -> rr64.
dwf_status g_true_residual(const Group& G, cudaStream_t st) {
  const int* skip = G.fl + FL_SKIP * G.nseg;
  void* const* f = G.f64;   // b, x, r, t1, t2, t3
  DWF_TRY(g_mpc(G, P64, f[1], f[3], f[4], f[5], false, skip, st));
  DWF_TRY(g_mpcdag(G, P64, f[5], f[4], f[2], nullptr, false, skip, st));
  return g_vop(G, P64, VOP_XMY_NORM, f[0], f[2], skip, FIN_STORE, G.sc + SC_RR64 * G.nseg, st);
}

// Starts (or restarts) the FP32 cycle of the problems with skip == 0 from their r64.
dwf_status g_cycle_start(const Group& G, bool first, cudaStream_t st) {
  const int* skip = G.fl + FL_SKIP * G.nseg;
  void** v = const_cast<void**>(G.f32);
  CastArgs c{};
  c.in = G.f64[2];
  c.out = v[2];
  c.Vp = G.Vp;
  c.Vhb = (int)G.Vp;
  c.Vhb_pad = (int)G.Vp;
  c.num = 1.0;
  c.out2 = first ? v[1] : nullptr;   // p = r at the very start
  c.stop = skip;
  c.tile_seg = G.tile_seg;
  c.segp = G.segp[0];
  c.red = gred(G, FIN_STORE);
  c.red.res = G.sc + SC_RHO * G.nseg;
  DWF_CUDA(launch_cast(P64, P32, c, G.Ls, st));
  DWF_TRY(g_vop(G, P32, VOP_ZERO, nullptr, v[0], skip, 0, nullptr, st));
  if (first) {
    VecArgs u{};
    u.p = v[1];
    u.u = v[3];
    u.Vp = G.Vp;
    u.Vhb = (int)G.Vp;
    u.Vhb_pad = (int)G.Vp;
    u.seg_cps = (int)G.ntiles;
    u.do_u = 1;
    u.stop = skip;
    u.tile_seg = G.tile_seg;
    u.segp = G.segp[1];
    DWF_CUDA(launch_vec(P32, u, G.Ls, st));
  }
  return DWF_OK;
}

dwf_status build_group(Batch& B, Group& G, const dwf_problem* pr) {
  cudaStream_t st = B.st;
  const int Ls = G.Ls;
  G.nseg = (int)G.ids.size();
  long tiles = 0;
  for (int q : G.ids) {
    Prob& P = B.probs[q];
    P.first_tile = tiles;
    P.ntiles = P.Vp / 32;
    tiles += P.ntiles;
  }
  G.ntiles = tiles;
  G.Vp = tiles * 32;
  const long Vp = G.Vp;
  // tables
  std::vector<uint32_t> nbr[2] = {std::vector<uint32_t>(8 * Vp, 0u), std::vector<uint32_t>(8 * Vp, 0u)};
  std::vector<int> lex[2] = {std::vector<int>(Vp, -1), std::vector<int>(Vp, -1)};
  std::vector<int> tseg(tiles);
  std::vector<long> loff(G.nseg);
  for (int k = 0; k < G.nseg; k++) {
    const Prob& P = B.probs[G.ids[k]];
    loff[k] = P.off_links;
    for (long t = 0; t < P.ntiles; t++) tseg[P.first_tile + t] = k;
    const int* d = P.dims;
    const long off = P.first_tile * 32;
    for (int par = 0; par < 2; par++) {
      for (long j = 0; j < P.Vh; j++) {
        const int hx = d[0] / 2;
        long r = j;
        const int jx = (int)(r % hx);
        r /= hx;
        int c[4];
        c[1] = (int)(r % d[1]);
        r /= d[1];
        c[2] = (int)(r % d[2]);
        c[3] = (int)(r / d[2]);
        c[0] = 2 * jx + ((par + c[1] + c[2] + c[3]) & 1);
        lex[par][off + j] = (int)(c[0] + (long)d[0] * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3])));
        for (int dd = 0; dd < 8; dd++) {
          int n[4] = {c[0], c[1], c[2], c[3]};
          const int mu = dd >> 1;
          n[mu] = (n[mu] + ((dd & 1) ? d[mu] - 1 : 1)) % d[mu];
          nbr[par][dd * Vp + off + j] = (uint32_t)(off + plain_index(d, n));
        }
      }
    }
  }
  for (int par = 0; par < 2; par++) {
    DWF_TRY(G.alloc(&G.nbr[par], nbr[par].size() * 4));
    DWF_TRY(G.alloc(&G.lex[par], lex[par].size() * 4));
    DWF_CUDA(cudaMemcpy(G.nbr[par], nbr[par].data(), nbr[par].size() * 4, cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(G.lex[par], lex[par].data(), lex[par].size() * 4, cudaMemcpyHostToDevice));
  }
  DWF_TRY(G.alloc(&G.tile_seg, tseg.size() * 4));
  DWF_CUDA(cudaMemcpy(G.tile_seg, tseg.data(), tseg.size() * 4, cudaMemcpyHostToDevice));
  long* dloff;
  DWF_TRY(G.alloc(&dloff, loff.size() * sizeof(long)));
  DWF_CUDA(cudaMemcpy(dloff, loff.data(), loff.size() * sizeof(long), cudaMemcpyHostToDevice));
  // per-problem fifth-dimension matrices (explicit D+: the pre-op always runs)
  const size_t msz = 3 * 2 * (size_t)Ls * Ls;
  std::vector<double> m64(msz * G.nseg);
  std::vector<float> m32(msz * G.nseg);
  std::vector<BatchSeg> seg64(G.nseg), seg32(G.nseg);
  DWF_TRY(G.alloc(&G.mats[0], m64.size() * sizeof(double)));
  DWF_TRY(G.alloc(&G.mats[1], m32.size() * sizeof(float)));
  for (int k = 0; k < G.nseg; k++) {
    const Prob& P = B.probs[G.ids[k]];
    std::vector<double> dpm5i, m5idpt, dpt;
    double la, lb;
    if (!fifth_dim_matrices(Ls, P.M5, P.mf, P.b, P.c, dpm5i, m5idpt, dpt, &la, &lb))
      return set_error(DWF_ERR_ARG, "batched solver: M5op is singular");
    if (P.c == 0.0)
      for (auto& x : dpm5i) x /= P.b;   // undo the absorbed pre-op factor
    const std::vector<double>* src[3] = {&dpm5i, &m5idpt, &dpt};
    for (int w = 0; w < 3; w++)
      for (int i = 0; i < 2 * Ls * Ls; i++) {
        m64[k * msz + w * 2 * Ls * Ls + i] = (*src[w])[i];
        m32[k * msz + w * 2 * Ls * Ls + i] = (float)(*src[w])[i];
      }
    for (int pr2 = 0; pr2 < 2; pr2++) {
      BatchSeg& S = pr2 ? seg32[k] : seg64[k];
      for (int w = 0; w < 3; w++)
        S.mat[w] = pr2 ? (const void*)((float*)G.mats[1] + k * msz + w * 2 * Ls * Ls)
                       : (const void*)((double*)G.mats[0] + k * msz + w * 2 * Ls * Ls);
      if (!(std::fabs(lb) < std::fabs(la))) G.post_struct = 0;
      S.l_alpha = la;
      S.l_beta = lb;
      S.mf = P.mf;
      S.db = P.b;
      S.dc = P.c;
      S.k64 = make_coef5<double>(la, lb, P.mf, P.b, P.c, 1.0, Ls);
      S.k32 = make_coef5<float>(la, lb, P.mf, P.b, P.c, 1.0, Ls);
      S.Vh = (int)P.Vh;
      S.first_tile = (int)P.first_tile;
      S.ntiles = (int)P.ntiles;
    }
  }
  DWF_CUDA(cudaMemcpy(G.mats[0], m64.data(), m64.size() * sizeof(double), cudaMemcpyHostToDevice));
  DWF_CUDA(cudaMemcpy(G.mats[1], m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice));
  for (int pr2 = 0; pr2 < 2; pr2++) {
    DWF_TRY(G.alloc(&G.segp[pr2], G.nseg * sizeof(BatchSeg)));
    DWF_CUDA(cudaMemcpy(G.segp[pr2], (pr2 ? seg32 : seg64).data(), G.nseg * sizeof(BatchSeg),
                        cudaMemcpyHostToDevice));
  }
  // links in FP64 and FP32
  for (int pi = 0; pi < 2; pi++) {
    const int prec = pi ? P32 : P64;
    const int nchl = prec == P64 ? 9 : 5;
    for (int par = 0; par < 2; par++) {
      DWF_TRY(G.alloc(&G.links[pi][par], (size_t)8 * nchl * 16 * Vp));
      dim3 grid((unsigned)((Vp + 127) / 128), 8), block(128);
      const double2* U = reinterpret_cast<const double2*>(B.staged_links);
      if (prec == P64)
        batch_pack_links_kernel<P64><<<grid, block, 0, st>>>(
            U, G.links[pi][par], G.nbr[par], G.lex[par], G.lex[1 - par], G.tile_seg, dloff, Vp);
      else
        batch_pack_links_kernel<P32><<<grid, block, 0, st>>>(
            U, G.links[pi][par], G.nbr[par], G.lex[par], G.lex[1 - par], G.tile_seg, dloff, Vp);
      DWF_CUDA(cudaGetLastError());
    }
  }
  // fields, scalars, flags, reduction scratch
  const size_t f64b = (size_t)Ls * Vp * 24 * 8, f32b = (size_t)Ls * Vp * 24 * 4;
  for (auto& f : G.f64) DWF_TRY(G.alloc(&f, f64b));
  for (auto& f : G.f32) DWF_TRY(G.alloc(&f, f32b));
  DWF_TRY(G.alloc(&G.sc, SC_N * G.nseg * sizeof(double)));
  DWF_TRY(G.alloc(&G.fl, FL_N * G.nseg * sizeof(int)));
  DWF_TRY(G.alloc(&G.counter, G.nseg * sizeof(unsigned)));
  DWF_TRY(G.alloc(&G.partial, (size_t)G.ntiles * sizeof(double)));
  DWF_TRY(G.alloc(&G.bar, sizeof(unsigned)));
  DWF_TRY(G.alloc(&G.err, sizeof(int)));
  DWF_CUDA(cudaMemsetAsync(G.err, 0, sizeof(int), st));
  DWF_CUDA(cudaMemsetAsync(G.sc, 0, SC_N * G.nseg * sizeof(double), st));
  DWF_CUDA(cudaMemsetAsync(G.fl, 0, FL_N * G.nseg * sizeof(int), st));
  DWF_CUDA(cudaMemsetAsync(G.counter, 0, G.nseg * sizeof(unsigned), st));
  DWF_CUDA(cudaMemsetAsync(G.f32[1], 0, f32b, st));
  // caller pointers (sources staged on the device if needed)
  std::vector<const double2*> srcs(G.nseg);
  std::vector<double2*> dsts(G.nseg);
  for (int k = 0; k < G.nseg; k++) {
    const int q = G.ids[k];
    const Prob& P = B.probs[q];
    const size_t ub = (size_t)Ls * P.Vh * 12 * 16;
    const void* phi = pr[q].phi;
    if (!is_device_ptr(phi)) {
      void* d;
      DWF_TRY(G.alloc(&d, ub));
      DWF_CUDA(cudaMemcpyAsync(d, phi, ub, cudaMemcpyHostToDevice, st));
      phi = d;
    }
    void* x = pr[q].x;
    if (!is_device_ptr(x)) DWF_TRY(G.alloc(&x, ub));
    srcs[k] = reinterpret_cast<const double2*>(phi);
    dsts[k] = reinterpret_cast<double2*>(x);
  }
  DWF_TRY(G.alloc(&G.srcs, G.nseg * sizeof(void*)));
  DWF_TRY(G.alloc(&G.dsts, G.nseg * sizeof(void*)));
  DWF_CUDA(cudaMemcpy(G.srcs, srcs.data(), G.nseg * sizeof(void*), cudaMemcpyHostToDevice));
  DWF_CUDA(cudaMemcpy(G.dsts, dsts.data(), G.nseg * sizeof(void*), cudaMemcpyHostToDevice));
  return DWF_OK;
}

// Autotuner: times stage A of the group for candidate persistent grid sizes (CTAs per SM) and
// keeps the fastest; results are cached per (Ls, tile count) for the process.
dwf_status autotune(Group& G, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, long>, int> cache;   // (device, Ls, tiles) -> grid
  int dev, sms;
  DWF_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, G.Ls, G.ntiles);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      G.grid = it->second;
      return DWF_OK;
    }
  }
  DWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cand[] = {1, 2, 3, 4, 0};
  cudaEvent_t e0, e1;
  DWF_CUDA(cudaEventCreate(&e0));
  DWF_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_grid = 0;
  for (int c : cand) {
    G.grid = c ? c * sms : 0;
    // the stage A launch of a CG step, with the problems' stop flags like the real launches
    // (the per-stage variant tuner never times launches that carry stop flags)
    StageArgs a = gbase(G, P32, 1, G.fl + FL_STOP * G.nseg);
    a.in = G.f32[3];
    a.out = G.f32[4];
    a.post = G.mats[1];
    a.post_which = 0;
    a.post_struct = G.post_struct;
    a.post_pre = 1.0;
    DWF_CUDA(launch_stage_prec(P32, a, G.Ls, false, false, st));   // warm
    DWF_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; r++) DWF_CUDA(launch_stage_prec(P32, a, G.Ls, false, false, st));
    DWF_CUDA(cudaEventRecord(e1, st));
    DWF_CUDA(cudaEventSynchronize(e1));
    float ms;
    DWF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_grid = G.grid;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  G.grid = best_grid;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best_grid;
  }
  return DWF_OK;
}

// The chunk form picked for a group, kept across calls: the same problem mix (Ls, sizes of
// the problems in order, and the DWF_BATCH_FORM restriction) reuses it instead of timing the
// candidates again.
struct ChunkChoice {
  int gather, grid;
};
std::mutex g_chunk_mu;
std::map<std::string, ChunkChoice> g_chunk_cache;

std::string chunk_key(const Batch& B, const Group& G, const char* form) {
  std::string k = std::to_string(G.Ls) + "|" + (form ? form : "") + "|";
  for (int q : G.ids) {
    const Prob& P = B.probs[q];
    for (int m = 0; m < 4; m++) k += std::to_string(P.dims[m]) + (m < 3 ? "x" : ",");
  }
  return k;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_batch_solve(int n, const dwf_problem* problems, double tol, int maxit,
                                      dwf_stats* per_solve, void* stream) {
  if (n <= 0 || !problems) return set_error(DWF_ERR_ARG, "no problems");
  if (!(tol > 0.0) || maxit < 0) return set_error(DWF_ERR_ARG, "bad tolerance or maxit");
  const auto t0 = std::chrono::steady_clock::now();
  Batch B;
  // all work runs on a private non-blocking stream (stream capture is not possible on the
  // legacy default stream), ordered after the caller's stream
  cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
  DWF_CUDA(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
  B.own_stream = true;
  {
    cudaEvent_t ev;
    DWF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DWF_CUDA(cudaEventRecord(ev, caller));
    DWF_CUDA(cudaStreamWaitEvent(B.st, ev, 0));
    cudaEventDestroy(ev);
  }
  long link_elems = 0;
  for (int i = 0; i < n; i++) {
    const dwf_problem& p = problems[i];
    Prob P{};
    for (int m = 0; m < 4; m++) {
      if (p.dims[m] < 2 || p.dims[m] % 2) return set_error(DWF_ERR_ARG, "dims must be even and >= 2");
      P.dims[m] = p.dims[m];
    }
    if (!(p.Ls == 4 || p.Ls == 6 || p.Ls == 8 || p.Ls == 10 || p.Ls == 12 || p.Ls == 16))
      return set_error(DWF_ERR_ARG, "Ls must be one of 4, 6, 8, 10, 12, 16");
    if (!p.links || !p.phi || !p.x) return set_error(DWF_ERR_ARG, "null field pointer");
    P.Ls = p.Ls;
    P.M5 = p.M5;
    P.mf = p.mf;
    P.b = p.b;
    P.c = p.c;
    P.V = (long)p.dims[0] * p.dims[1] * p.dims[2] * p.dims[3];
    P.Vh = P.V / 2;
    P.Vp = (P.Vh + 31) / 32 * 32;
    P.off_links = link_elems;
    link_elems += P.V * 4 * 9;
    B.probs.push_back(P);
  }
  // stage every problem's links into one device buffer
  {
    void* d;
    if (cudaMalloc(&d, (size_t)link_elems * 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(DWF_ERR_NOMEM, "batched solver: links staging allocation failed");
    }
    B.owned.push_back(d);
    B.staged_links = static_cast<double*>(d);
    for (int i = 0; i < n; i++)
      DWF_CUDA(cudaMemcpyAsync(B.staged_links + 2 * B.probs[i].off_links, problems[i].links,
                               (size_t)B.probs[i].V * 4 * 9 * 16, cudaMemcpyDefault, B.st));
  }
  std::map<int, std::vector<int>> by_ls;
  for (int i = 0; i < n; i++) by_ls[B.probs[i].Ls].push_back(i);
  for (auto& kv : by_ls) {
    auto G = std::make_unique<Group>();
    G->Ls = kv.first;
    G->ids = kv.second;
    DWF_TRY(build_group(B, *G, problems));
    B.groups.push_back(std::move(G));
  }
  // initial state: b64 = phi, x64 = 0, r64 = b, bb = ||b||^2, stop2 = max(delta^2, tol^2) bb
  std::vector<std::vector<double>> bb(B.groups.size());
  for (size_t gi = 0; gi < B.groups.size(); gi++) {
    Group& G = *B.groups[gi];
    dim3 grid((unsigned)((G.Vp + 127) / 128), G.Ls), block(128);
    batch_move_kernel<<<grid, block, 0, B.st>>>(G.srcs, G.dsts, (double2*)G.f64[0], G.tile_seg,
                                                 G.segp[0], nullptr, G.Vp, 1);
    DWF_CUDA(cudaGetLastError());
    DWF_TRY(g_vop(G, P64, VOP_ZERO, nullptr, G.f64[1], nullptr, 0, nullptr, B.st));
    DWF_TRY(g_vop(G, P64, VOP_COPY, G.f64[0], G.f64[2], nullptr, 0, nullptr, B.st));
    DWF_TRY(g_vop(G, P64, VOP_NORM, G.f64[2], nullptr, nullptr, FIN_STORE,
                  G.sc + SC_BB * G.nseg, B.st));
    bb[gi].resize(G.nseg);
    DWF_CUDA(cudaMemcpyAsync(bb[gi].data(), G.sc + SC_BB * G.nseg, G.nseg * sizeof(double),
                             cudaMemcpyDeviceToHost, B.st));
  }
  DWF_CUDA(cudaStreamSynchronize(B.st));
  const double delta = 0.1;
  std::vector<std::vector<double>> rr(B.groups.size()), stop2h(B.groups.size());
  std::vector<std::vector<int>> done(B.groups.size()), iters(B.groups.size()),
      rus(B.groups.size());
  for (size_t gi = 0; gi < B.groups.size(); gi++) {
    Group& G = *B.groups[gi];
    rr[gi] = bb[gi];
    done[gi].assign(G.nseg, 0);
    iters[gi].assign(G.nseg, 0);
    rus[gi].assign(G.nseg, 0);
    std::vector<double>& stop2 = stop2h[gi];
    stop2.resize(G.nseg);
    for (int k = 0; k < G.nseg; k++) {
      stop2[k] = std::max(delta * delta * rr[gi][k], tol * tol * bb[gi][k]);
      if (!(bb[gi][k] > 0.0)) done[gi][k] = 1;
    }
    DWF_CUDA(cudaMemcpyAsync(G.sc + SC_STOP2 * G.nseg, stop2.data(), G.nseg * sizeof(double),
                             cudaMemcpyHostToDevice, B.st));
    std::vector<int> fl(FL_N * G.nseg, 0);
    for (int k = 0; k < G.nseg; k++) fl[FL_STOP * G.nseg + k] = fl[FL_SKIP * G.nseg + k] = done[gi][k];
    DWF_CUDA(cudaMemcpyAsync(G.fl, fl.data(), fl.size() * sizeof(int), cudaMemcpyHostToDevice, B.st));
    DWF_TRY(g_cycle_start(G, true, B.st));
    DWF_TRY(autotune(G, B.st));
  }
  DWF_CUDA(cudaStreamSynchronize(B.st));

  // a chunk of CG steps of every group: one persistent launch per group, or one launch per
  // stage and update (g_cg_step, each stage with its own tuned variant).  The first chunks time
  // the candidates (the stage launches; the persistent launch with a grid of 1 or 2 CTAs per
  // SM or the largest co-resident grid, links read directly or staged by TMA bulk copies); the
  // fastest of each group is then captured once in a CUDA graph and replayed.  Groups whose
  // fifth-dimension post cannot use the recurrences keep the stage launches.
  const int chunk = 16;
  int dev = 0, nsm = 1;
  DWF_CUDA(cudaGetDevice(&dev));
  DWF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (const char* wl = getenv("DWF_WAIT_LIMIT_US")) {
    const double us = atof(wl);
    if (us >= 1.0 && us <= 1e7) B.wait_ns = (unsigned long long)(us * 1000.0);
  }
  const unsigned long long wait_ns = B.wait_ns;
  struct Cand {
    int gather, grid;
  };
  std::vector<std::vector<Cand>> cands(B.groups.size());
  std::vector<std::string> keys(B.groups.size());
  for (size_t gi = 0; gi < B.groups.size(); gi++) {
    Group& G = *B.groups[gi];
    if (!G.post_struct) continue;
    // DWF_BATCH_FORM=stages|persistent restricts the candidates to one form
    const char* form = getenv("DWF_BATCH_FORM");
    const bool only_stages = form && strcmp(form, "stages") == 0;
    const bool only_persistent = form && strcmp(form, "persistent") == 0;
    keys[gi] = chunk_key(B, G, form);
    {
      std::lock_guard<std::mutex> lk(g_chunk_mu);
      auto it = g_chunk_cache.find(keys[gi]);
      if (it != g_chunk_cache.end()) {   // decided by an earlier call on this problem mix
        G.sgather = it->second.gather;
        G.sgrid = it->second.grid;
        continue;
      }
    }
    if (!only_persistent) cands[gi].push_back({-1, 0});   // one launch per stage (gather -1)
    if (only_stages) continue;
    BatchStepArgs ba;
    g_step_args(G, chunk, wait_ns, ba);
    for (int gather : {G_REG, G_TMA}) {
      int cap = 0;
      DWF_CUDA(batch_steps_launch(ba, G.Ls, gather, 0, &cap, nsm, B.st, true));
      std::vector<int> grids;
      for (int per : {1, 2}) if (per * nsm <= cap) grids.push_back(per * nsm);
      if (cap > 2 * nsm) grids.push_back(cap);
      for (int g : grids) cands[gi].push_back({gather, (int)std::min<long>(g, G.ntiles)});
    }

  }
  size_t ntune = 0;
  for (auto& c : cands) ntune = std::max(ntune, c.size());
  std::vector<std::vector<float>> tuned(B.groups.size());
  cudaEvent_t tev[2];
  DWF_CUDA(cudaEventCreate(&tev[0]));
  DWF_CUDA(cudaEventCreate(&tev[1]));
  auto launch_chunk = [&](Group& G, int gather, int grid) -> dwf_status {
    BatchStepArgs ba;
    g_step_args(G, chunk, wait_ns, ba);
    DWF_CUDA(cudaMemsetAsync(G.bar, 0, sizeof(unsigned), B.st));
    int cap = 0;
    DWF_CUDA(batch_steps_launch(ba, G.Ls, gather, grid, &cap, nsm, B.st, false));
    return DWF_OK;
  };
  auto stage_chunk = [&](Group& G) -> dwf_status {
    for (int k = 0; k < chunk; k++) DWF_TRY(g_cg_step(G, B.st));
    return DWF_OK;
  };
  size_t tune_round = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // a first un-captured step of the stage path sets its kernels' attributes
  for (auto& G : B.groups) DWF_TRY(g_cg_step(*G, B.st));
  auto capture = [&]() -> dwf_status {
    DWF_CUDA(cudaStreamSynchronize(B.st));
    DWF_CUDA(cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal));
    for (auto& Gp : B.groups) {
      Group& G = *Gp;
      dwf_status s = (G.post_struct && G.sgather >= 0) ? launch_chunk(G, G.sgather, G.sgrid)
                                                        : stage_chunk(G);
      if (s != DWF_OK) {
        cudaStreamEndCapture(B.st, &graph);
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        return s;
      }
    }
    DWF_CUDA(cudaStreamEndCapture(B.st, &graph));
    DWF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    return DWF_OK;
  };
  if (ntune == 0) DWF_TRY(capture());
  // one chunk of every group: a tuning round (timed launches of the next candidate) or the
  // captured graph
  auto run_chunk = [&]() -> dwf_status {
    if (tune_round >= ntune) {
      DWF_CUDA(cudaGraphLaunch(exec, B.st));
      return DWF_OK;
    }
    for (size_t gi = 0; gi < B.groups.size(); gi++) {
      Group& G = *B.groups[gi];
      if (!G.post_struct || cands[gi].empty()) {   // stage launches only, or decided earlier
        if (G.post_struct && G.sgather >= 0) DWF_TRY(launch_chunk(G, G.sgather, G.sgrid));
        else DWF_TRY(stage_chunk(G));
        continue;
      }
      const Cand& c = cands[gi][std::min(tune_round, cands[gi].size() - 1)];
      DWF_CUDA(cudaEventRecord(tev[0], B.st));
      if (c.gather < 0) DWF_TRY(stage_chunk(G));
      else DWF_TRY(launch_chunk(G, c.gather, c.grid));
      DWF_CUDA(cudaEventRecord(tev[1], B.st));
      DWF_CUDA(cudaEventSynchronize(tev[1]));
      float ms = 0.f;
      DWF_CUDA(cudaEventElapsedTime(&ms, tev[0], tev[1]));
      if (tune_round < cands[gi].size()) tuned[gi].push_back(ms);
    }
    if (++tune_round == ntune) {
      for (size_t gi = 0; gi < B.groups.size(); gi++) {
        Group& G = *B.groups[gi];
        if (!G.post_struct || cands[gi].empty()) continue;
        size_t best = 0;
        for (size_t k = 1; k < tuned[gi].size(); k++)
          if (tuned[gi][k] < tuned[gi][best]) best = k;
        G.sgather = cands[gi][best].gather;
        G.sgrid = cands[gi][best].grid;
        {
          std::lock_guard<std::mutex> lk(g_chunk_mu);
          g_chunk_cache[keys[gi]] = {G.sgather, G.sgrid};
        }
        if (getenv("DWF_TUNE_LOG")) {
          fprintf(stderr, "dwf tune batch Ls%d tiles %ld:", G.Ls, G.ntiles);
          for (size_t k = 0; k < tuned[gi].size(); k++)
            fprintf(stderr, " %s[gather%d grid%d %.2fms]", k == best ? "*" : "",
                    cands[gi][k].gather, cands[gi][k].grid, tuned[gi][k]);
          fprintf(stderr, "\n");
        }
      }
      DWF_TRY(capture());
    }
    return DWF_OK;
  };

  int total_steps = 0;
  dwf_status status = DWF_OK;
  while (true) {
    DWF_TRY(run_chunk());
    total_steps += chunk;
    bool all_done = true, any_ru = false;
    for (size_t gi = 0; gi < B.groups.size(); gi++) {
      Group& G = *B.groups[gi];
      std::vector<int> fl(FL_N * G.nseg);
      DWF_CUDA(cudaMemcpyAsync(fl.data(), G.fl, fl.size() * sizeof(int), cudaMemcpyDeviceToHost, B.st));
      DWF_CUDA(cudaStreamSynchronize(B.st));
      std::vector<int> skip(G.nseg, 1);
      bool ru = false;
      for (int k = 0; k < G.nseg; k++) {
        if (done[gi][k]) continue;
        const int it = iters[gi][k] + fl[FL_ITER * G.nseg + k];
        if (fl[FL_STOP * G.nseg + k] || it >= maxit) {
          skip[k] = 0;
          ru = true;
        }
      }
      if (ru) {
        any_ru = true;
        // x64 += x32, r64 = b - A64 x64 for the selected problems
        DWF_CUDA(cudaMemcpyAsync(G.fl + FL_SKIP * G.nseg, skip.data(), G.nseg * sizeof(int),
                                 cudaMemcpyHostToDevice, B.st));
        DWF_TRY(g_vop(G, P64, VOP_ADD_CAST, G.f32[0], G.f64[1], G.fl + FL_SKIP * G.nseg, 0,
                      nullptr, B.st, P32));
        DWF_TRY(g_true_residual(G, B.st));
        std::vector<double> r64(G.nseg);
        DWF_CUDA(cudaMemcpyAsync(r64.data(), G.sc + SC_RR64 * G.nseg, G.nseg * sizeof(double),
                                 cudaMemcpyDeviceToHost, B.st));
        DWF_CUDA(cudaStreamSynchronize(B.st));
        std::vector<double>& stop2 = stop2h[gi];
        for (int k = 0; k < G.nseg; k++) {
          if (skip[k]) continue;
          iters[gi][k] += fl[FL_ITER * G.nseg + k];
          fl[FL_ITER * G.nseg + k] = 0;
          rus[gi][k]++;
          rr[gi][k] = r64[k];
          if (r64[k] <= tol * tol * bb[gi][k] || iters[gi][k] >= maxit || !std::isfinite(r64[k])) {
            done[gi][k] = 1;
            fl[FL_STOP * G.nseg + k] = 1;
            skip[k] = 1;   // no restart
          } else {
            fl[FL_STOP * G.nseg + k] = 0;
            fl[FL_CONV * G.nseg + k] = 0;
            stop2[k] = std::max(delta * delta * r64[k], tol * tol * bb[gi][k]);
          }
        }
        for (int k = 0; k < G.nseg; k++) fl[FL_SKIP * G.nseg + k] = skip[k];
        DWF_CUDA(cudaMemcpyAsync(G.sc + SC_STOP2 * G.nseg, stop2.data(), G.nseg * sizeof(double),
                                 cudaMemcpyHostToDevice, B.st));
        DWF_CUDA(cudaMemcpyAsync(G.fl, fl.data(), fl.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 B.st));
        // restart the FP32 cycle of the problems that continue (p is kept)
        DWF_TRY(g_cycle_start(G, false, B.st));
        DWF_CUDA(cudaStreamSynchronize(B.st));
      }
      for (int k = 0; k < G.nseg; k++) all_done = all_done && done[gi][k];
    }
    (void)any_ru;
    if (all_done) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(tev[0]);
  cudaEventDestroy(tev[1]);
  for (auto& Gp : B.groups) {   // a bounded device wait that gave up invalidates the solve
    int e = 0;
    DWF_CUDA(cudaMemcpyAsync(&e, Gp->err, sizeof(int), cudaMemcpyDeviceToHost, B.st));
    DWF_CUDA(cudaStreamSynchronize(B.st));
    if (e) return set_error(DWF_ERR_TIMEOUT, "batched solver: a bounded device wait gave up");
  }
  // solutions out
  for (size_t gi = 0; gi < B.groups.size(); gi++) {
    Group& G = *B.groups[gi];
    dim3 grid((unsigned)((G.Vp + 127) / 128), G.Ls), block(128);
    batch_move_kernel<<<grid, block, 0, B.st>>>(G.srcs, G.dsts, (double2*)G.f64[1], G.tile_seg,
                                                 G.segp[0], nullptr, G.Vp, 0);
    DWF_CUDA(cudaGetLastError());
  }
  DWF_CUDA(cudaStreamSynchronize(B.st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (size_t gi = 0; gi < B.groups.size(); gi++) {
    Group& G = *B.groups[gi];
    std::vector<double2*> dsts(G.nseg);
    DWF_CUDA(cudaMemcpyAsync(dsts.data(), G.dsts, G.nseg * sizeof(void*), cudaMemcpyDeviceToHost,
                             B.st));
    DWF_CUDA(cudaStreamSynchronize(B.st));
    for (int k = 0; k < G.nseg; k++) {
      const int q = G.ids[k];
      if (!is_device_ptr(problems[q].x)) {
        const size_t ub = (size_t)G.Ls * B.probs[q].Vh * 12 * 16;
        DWF_CUDA(cudaMemcpyAsync(problems[q].x, dsts[k], ub, cudaMemcpyDeviceToHost, B.st));
        DWF_CUDA(cudaStreamSynchronize(B.st));
      }
      const double res = std::sqrt(rr[gi][k] / bb[gi][k]);
      if (!(res <= tol) && bb[gi][k] > 0.0) status = DWF_ERR_NOT_CONVERGED;
      if (per_solve) {
        dwf_stats& s = per_solve[q];
        s.iterations = iters[gi][k];
        s.inner_iterations = 0;
        s.reliable_updates = rus[gi][k];
        s.operator_applications = iters[gi][k] + rus[gi][k];
        s.true_residual = bb[gi][k] > 0.0 ? res : 0.0;
        s.seconds = secs;
        s.history_len = 0;
      }
    }
  }
  (void)total_steps;
  if (status != DWF_OK) set_error(status, "a batched problem did not reach the tolerance");
  return status;
}
