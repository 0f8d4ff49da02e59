// Host-side internals of libdwf: geometry of a site ordering, packed layouts, kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dwf.h"
#include "dwf_device.cuh"
#include "stage.cuh"

namespace dwf {

// Thread-local error message; set_error returns the status for convenience.
dwf_status set_error(dwf_status st, const std::string& msg);
dwf_status cuda_error(cudaError_t e, const char* what);

#define DWF_CUDA(call)                                          \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return cuda_error(_e, #call);        \
  } while (0)

#define DWF_TRY(call)                                           \
  do {                                                          \
    dwf_status _s = (call);                                     \
    if (_s != DWF_OK) return _s;                                \
  } while (0)

// A site ordering: the lattice is cut into blocks B (B = L gives one block, i.e. plain
// checkerboard order); sites of one parity are stored block after block, each block padded
// to a multiple of 32 sites.  Index of a parity-p site: blk * Vhb_pad + j,
// j = (lx/2) + (Bx/2) * (ly + By * (lz + Bz * lt)) with (lx, ly, lz, lt) block-local.
struct Geom {
  int L[4];
  int B[4];
  int nb[4];
  int nblocks;
  int Vhb;       // sites of one parity per block
  int Vhb_pad;   // padded to a multiple of 32
  long Vp;       // nblocks * Vhb_pad
  long V;        // full volume
  int Ls;
  bool same(const int* blk) const {
    return B[0] == blk[0] && B[1] == blk[1] && B[2] == blk[2] && B[3] == blk[3];
  }
};

// Halo of every block for the exact block operator P_s A P_s: the odd sites one hop outside
// the block and the even sites up to two hops outside (Mpc P_s v is supported on the block
// plus its even halo).  Each block owns its own halo arrays, padded to 32 sites.
struct Halo {
  int Ho_b = 0, Ho_pad = 0, He_b = 0, He_pad = 0;
  long Ho_tot = 0, He_tot = 0;
  uint32_t* nbr_be = nullptr;  // [8][Vp] block even -> odd (in block | HALO odd halo)
  uint32_t* nbr_bo = nullptr;  // [8][Vp] block odd -> even (in block | HALO even halo)
  uint32_t* nbr_ho = nullptr;  // [8][Ho_tot] odd halo -> even (in block | HALO | FACE absent)
  uint32_t* nbr_he = nullptr;  // [8][He_tot] even halo -> odd (in block | HALO | FACE absent)
  int* ls_ho = nullptr;        // [Ho_tot] odd halo site -> its odd index (links)
  int* ls_he = nullptr;        // [He_tot] even halo site -> its even index (links)
  void* links_ho[4] = {};      // per precision: links of the odd halo sites, contiguous
  void* links_he[4] = {};      // per precision: links of the even halo sites, contiguous
  ~Halo();
};

struct SimdArgs;

// Block-SIMD geometry of the local solves for one block shape and one local operator (see
// local_kernel.cuh): the block-relative positions of E = BE ++ HE and O = BO ++ HO, their
// neighbour tables, per-phase schedules, element <-> outer-site maps and packed links.
struct SimdLocal {
  bool exact = false;
  int nb = 0, NB = 0, ngroups = 0;
  int nbk[4] = {1, 1, 1, 1};  // blocks per direction
  int nBE = 0, nE = 0, nO = 0;
  long sB = 0, sE = 0, sO = 0;
  uint32_t* nbrE = nullptr;   // [nE][8] -> O position or SIMD_ABSENT
  uint32_t* nbrO = nullptr;   // [nO][8] -> E position or SIMD_ABSENT
  uint32_t* sch = nullptr;    // P1 (nO) | P2 (nE) | P3 (nO) | P4 (nBE) schedules
  int nsch[4] = {0, 0, 0, 0};
  long sch_off[4] = {0, 0, 0, 0};
  int* lexE = nullptr;        // [sE] element -> lexicographic site (-1: none)
  int* lexO = nullptr;        // [sO]
  int* fwd = nullptr;         // [sB] BE element -> whole-lattice even index (-1: none)
  int* inv = nullptr;         // [V/2 rounded to 32] whole-lattice even index -> BE element
  void* linksE[4] = {};
  void* linksO[4] = {};
  bool links_valid[4] = {false, false, false, false};
  unsigned* ctr = nullptr;    // barrier counters
  double* partial = nullptr;
  int cap_slots = 0, cap_C = 0;
  // launch-variant tuner per storage precision: -1 undecided; events of the timed calls
  int tune_chosen[4] = {-1, -1, -1, -1};
  int tune_next[4] = {0, 0, 0, 0};
  cudaEvent_t tune_ev[4][24] = {};
  ~SimdLocal();
};

// Device tables and packed links of one site ordering.
struct Layout {
  std::unique_ptr<SimdLocal> simd[2];      // [exact]: local solves in the block-SIMD layout
  std::unique_ptr<Halo> halo;              // built on demand (exact block operator)
  Geom g;
  uint32_t* nbr[2] = {nullptr, nullptr};   // [8][Vp] per output parity
  int* lex[2] = {nullptr, nullptr};        // internal index -> lexicographic site (-1 = pad)
  int* cb_even = nullptr;                  // internal even index -> caller even-half index
  int* cb_inv = nullptr;                   // caller even-half index -> internal even index
                                           // ([V/2 rounded up to 32], -1 = pad)
  void* links[4][2] = {};                  // [precision][parity] packed links, lazily built
  bool links_valid[4] = {false, false, false, false};
  ~Layout();
};

// Per-chirality Ls x Ls matrices of the fifth dimension (double and float copies).
struct Matrices {
  // host copies in double, [2][Ls][Ls]
  std::vector<double> dp, dpt, dpm5i, m5idpt, m5, m5t;
  // device copies: [which][precision class: 0 double, 1 float]
  void* d_dpm5i[2] = {};   // D+ M5op^-1 (post of stage A)
  void* d_m5idpt[2] = {};  // M5op^-dag D+^dag (post of stage A^dag)
  void* d_dpt[2] = {};     // D+^dag (post of stage B^dag and of D^dag)
  void* d_dp[2] = {};      // D+ (pre-op)
  // FP16 16x16 tensor-core operands (core-matrix layout, [2 chiralities]) of
  // {D+ M5op^-1, M5op^-dag D+^dag, D+^dag}
  void* d_post_h[3] = {};
  bool use_tc = true;
  // how the stages apply the dense fifth-dimension post matrices: 0 auto (recurrences for
  // FP32/FP64, the faster of recurrences and tensor cores for FP16/BF16), 1 matrices only
  // (tensor cores for FP16/BF16), 2 recurrences only; recurrences need |beta/alpha| < 1
  int post_mode = 0;
  bool struct_ok = false;
  double m5_alpha = 0, m5_beta = 0;  // M5op = alpha + beta K
  bool dplus_trivial = true;         // c == 0 (D+ = b)
};

struct Workspace;

// Event-based per-kernel profiler of a handle (off by default).
struct Profiler {
  bool on = false;
  struct Rec {
    int cls;
    double bytes, flops;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  size_t used = 0;
  int class_id(const std::string& n) {
    for (size_t i = 0; i < names.size(); i++)
      if (names[i] == n) return (int)i;
    names.push_back(n);
    return (int)names.size() - 1;
  }
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// RAII bracket of one launch: records the start event at construction and the stop event
// (with the launch's algorithmic bytes) at destruction.
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  Profiler::Rec r{};
  ProfScope(Profiler* prof, cudaStream_t s, const char* name, double bytes, double flops)
      : p(prof && prof->on ? prof : nullptr), st(s) {
    if (!p) return;
    r.cls = p->class_id(name);
    r.bytes = bytes;
    r.flops = flops;
    r.a = p->ev();
    r.b = p->ev();
    cudaEventRecord(r.a, st);
  }
  ~ProfScope() {
    if (!p) return;
    cudaEventRecord(r.b, st);
    p->recs.push_back(r);
  }
};

inline const char* prec_name(int p) {
  return p == 0 ? "f64" : p == 1 ? "f32" : p == 2 ? "f16" : "bf16";
}

}  // namespace dwf

struct dwf_ctx {
  int dims[4];
  int Ls;
  double M5, mf, b, c;
  cudaStream_t stream;
  int device;
  double* links_c128 = nullptr;  // device copy of the caller links
  dwf::Matrices mats;
  std::vector<std::unique_ptr<dwf::Layout>> layouts;
  std::unique_ptr<dwf::Workspace> ws;
  // per-handle device scratch for reductions
  double* red_partial = nullptr;
  size_t red_partial_len = 0;
  unsigned* red_counter = nullptr;
  size_t red_counter_len = 0;
  double* scal = nullptr;   // device scalars (see Scalars in solvers)
  size_t scal_len = 0;
  double* h_pinned = nullptr;  // pinned host mirror for scalar reads
  int* dev_err = nullptr;      // set by a bounded device wait that gave up
  unsigned long long wait_ns = 0;  // limit of bounded device waits (0: the kernels' 10 ms)
  int wait_probe = 0;              // failure-detection test switch (see dwf_set_option)
  dwf::Profiler prof;
};

namespace dwf {

// ---- layouts and packing (pack.cu) ----
dwf_status get_layout(dwf_ctx* h, const int block[4], Layout** out);
dwf_status ensure_links(dwf_ctx* h, Layout* lay, int prec);
dwf_status ensure_halo(dwf_ctx* h, Layout* lay);
dwf_status build_matrices(dwf_ctx* h);
// Host copies ([2][Ls][Ls] each, double) of D+ M5op^-1 (times b when c = 0, absorbing the
// pre-op), M5op^-dag D+^dag and D+^dag, and M5op = alpha + beta K.
bool fifth_dim_matrices(int Ls, double M5, double mf, double b, double c,
                        std::vector<double>& dpm5i, std::vector<double>& m5idpt,
                        std::vector<double>& dpt, double* alpha, double* beta);

// Field sizes in bytes.
inline size_t real_bytes(int prec) { return prec == P64 ? 8 : prec == P32 ? 4 : 2; }
inline size_t field_bytes(const Geom& g, int prec) {
  return (size_t)g.Ls * (size_t)g.Vp * 24 * real_bytes(prec);
}

// Caller even-half c128 (device) <-> internal even field of precision prec.
// scale: multiplies on pack, divides on unpack (FP16/BF16 range control).
dwf_status pack_even(dwf_ctx* h, Layout* lay, const void* src_c128, void* dst, int prec,
                     double scale);
dwf_status unpack_even(dwf_ctx* h, Layout* lay, const void* src, int prec, void* dst_c128,
                       double scale);
// Caller full c128 <-> internal (even, odd) fields.
dwf_status pack_full(dwf_ctx* h, Layout* lay, const void* src_c128, void* dst_even,
                     void* dst_odd, int prec);
dwf_status unpack_full(dwf_ctx* h, Layout* lay, const void* src_even, const void* src_odd,
                       int prec, void* dst_c128);

// ---- stage kernels (stage_ls.cu per precision, Ls and dag; stage_dispatch.cu) ----
template <int P, int LS, bool DAG>
cudaError_t stage_dispatch_ls(const StageArgs& a, bool blocked, cudaStream_t st);
cudaError_t launch_stage_prec(int prec, const StageArgs& a, int Ls, bool dag, bool blocked,
                              cudaStream_t st);

// ---- block-SIMD local solves (local_solve.cu, local_p.cu) ----
dwf_status ensure_simd(dwf_ctx* h, Layout* lay, bool exact, SimdLocal** out);
// Runs the l local CG iterations of every block from a zero guess on r_local = f r_outer,
// f = sqrt(num / *den) (num when den is null); the solution is left in the BE field `x`
// (element layout; S->inv maps whole-lattice even sites to elements).  One cooperative launch.
struct SimdFields {
  void *x, *p, *u, *r, *t, *y;
};
// ncol > 1: only the blocks of colour col solve (the others return x = 0): one colour of a
// multiplicative Schwarz sweep (colours as in dwf_ms_solve).
dwf_status simd_local_solve(dwf_ctx* h, SimdLocal* S, int prec, int l, const void* r_outer,
                            int prec_outer, long Vp_outer, double num, const double* den,
                            const SimdFields& F, int ncol = 1, int col = 0);
// True once the local solver's launch variant for this storage precision is fixed (timed by
// the tuner, forced by DWF_LOCAL_VARIANT, or FP64's single variant).
bool simd_variant_decided(const SimdLocal* S, int prec);
template <int P>
cudaError_t simd_launch_p(const SimdArgs& a, int Ls, int v, int* grid_cap, int nsm, cudaStream_t st,
                          bool query);

// ---- vector kernels (blas.cu) ----
struct VecArgs {
  void* x;            // x += alpha * p         (if do_x)
  void* p;            // p = r + beta * p       (if do_p)
  const void* r;
  // z_src (nullable): read r as z = f * z_src[z_map[site]] instead, z_src a field of
  // precision z_prec and site stride z_vp in another site order (z_map nullable: same order),
  // f = 1 / sqrt(z_num / *z_den) (1 / z_num without z_den): the preconditioner's output is
  // used without being stored in this precision first
  const void* z_src;
  int z_prec;
  const int* z_map;
  long z_vp;
  double z_num;
  const double* z_den;
  void* u;            // u = (db + dc K) p_new  (if do_u)
  long Vp;
  int Vhb, Vhb_pad;
  const double* alpha;  // per segment
  const double* beta;   // per segment
  int seg_cps;          // CTAs per scalar segment
  int do_x, do_p, do_u;
  double db, dc, mf;
  const int* stop;
  RedArgs red;          // with red.partial != nullptr: grid completion + finalize
  int* stop_out;        // set *stop_out = *conv_in in the finalize (nullable)
  const int* conv_in;
  int* iter;            // incremented in the finalize (nullable)
  const int* tile_seg;  // batched mode (nullable): per-problem stop/iter/scalars and D+
  const BatchSeg* segp;
};
cudaError_t launch_vec(int prec, const VecArgs& a, int Ls, cudaStream_t st);

// ---- batched CG steps in one persistent launch (batch_steps.cu) ----
// A, B, Ad, Bd: the four stage launches of a CG step on A = Mpc^dag Mpc (finished with
// finish_stage_args), U: the update; nsteps steps per launch; bar: barrier counter, zero at
// launch.
struct BatchStepArgs {
  StageArgs A, B, Ad, Bd;
  VecArgs U;
  long ntiles;
  int nsteps;
  unsigned* bar;
  unsigned long long wait_ns;
  int* err;
};
// query: *cap = the largest co-resident grid; otherwise a cooperative launch of `grid` CTAs.
// gather: G_REG or G_TMA (how the stages read their links).
cudaError_t batch_steps_launch(const BatchStepArgs& b, int Ls, int gather, int grid, int* cap,
                               int nsm, cudaStream_t st, bool query);

// Elementwise conversion out = in * f (f = sqrt(num / *den) if den else num), both fields of
// the same geometry, with an optional reduction of <dotv, out> (dotv in out's precision).
struct CastArgs {
  const void* in;
  void* out;
  long Vp;
  const int* in_map;     // nullable: out site i reads in site in_map[i] (-1: zero)
  long Vp_in;            // site stride of in when in_map is set
  int Vhb, Vhb_pad;
  double num;
  const double* den;     // nullable
  int invert;            // use 1/f
  const void* dotv;      // nullable
  void* out2;            // nullable: second copy of out
  void* out3;            // nullable: D+ out (Moebius pre-op of the stored out)
  double db, dc, mf;     // D+ = db + dc K, walls -mf (out3)
  float dbf, dcf, mff;   // the same in FP32
  const int* stop;
  RedArgs red;
  const int* tile_seg;   // batched mode (nullable)
  const BatchSeg* segp;
};
cudaError_t launch_cast(int pin, int pout, const CastArgs& a, int Ls, cudaStream_t st);

// Generic small vector ops on one precision.
enum VOp {
  VOP_ZERO = 0,      // y = 0
  VOP_COPY = 1,      // y = x
  VOP_AXPY = 2,      // y = y + a x          (a from device scalar *ap times sa)
  VOP_XMY_NORM = 3,  // y = x - y, reduce |y|^2
  VOP_NORM = 4,      // reduce |x|^2
  VOP_DOT = 5,       // reduce Re <x, y>
  VOP_ADD_CAST = 6   // y (P64) += x (other precision)   [reliable update]
};
struct VopArgs {
  int op;
  const void* x;
  void* y;
  long Vp;
  int Vhb, Vhb_pad;
  double sa;
  const double* ap;
  const int* stop;
  RedArgs red;
  const int* tile_seg;   // batched mode (nullable)
  const BatchSeg* segp;
};
cudaError_t launch_vop(int prec, int prec_x, const VopArgs& a, int Ls, cudaStream_t st);

// ---- helpers (api.cu) ----
dwf_status ensure_reduction(dwf_ctx* h, size_t partials, size_t counters);
RedArgs make_red(dwf_ctx* h, int cps, int op, double* res);
dwf_status stage_buffer(dwf_ctx* h, const char* name, const void* user, size_t bytes,
                        bool copy_in, void** dev);
dwf_status finish_output(dwf_ctx* h, void* user, const void* dev, size_t bytes);
dwf_status check_device_error(dwf_ctx* h);
bool is_device_ptr(const void* p);

}  // namespace dwf
