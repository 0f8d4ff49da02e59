// Host side of the block-SIMD local solves (Sec. 2.3, Eqs. 4-5): the block-relative site
// sets of one block shape, their neighbour tables and schedules, the packed links of every
// block's sites in the position-major element order, and the cooperative launch of the
// persistent kernel (local_kernel.cuh).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <vector>

#include "engine.h"
#include "local_kernel.cuh"

namespace dwf {

SimdLocal::~SimdLocal() {
  cudaFree(nbrE);
  cudaFree(nbrO);
  cudaFree(sch);
  cudaFree(lexE);
  cudaFree(lexO);
  cudaFree(fwd);
  cudaFree(inv);
  for (int p = 0; p < 4; p++) {
    cudaFree(linksE[p]);
    cudaFree(linksO[p]);
  }
  cudaFree(ctr);
  cudaFree(partial);
  for (auto& row : tune_ev)
    for (auto e : row)
      if (e) cudaEventDestroy(e);
}

namespace {

template <typename T>
dwf_status upload(const std::vector<T>& v, T** dst) {
  DWF_CUDA(cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty())
    DWF_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DWF_OK;
}

// Links of element e (site lex[e], -1: none) for the 8 hop directions: U_mu(x) forward,
// U_mu(x - mu)^dag backward, in the chunked [dir][chunk][element] layout.
template <int P>
__global__ void pack_simd_links_kernel(const double2* __restrict__ U, void* out,
                                       const int* __restrict__ lex, long n, int X, int Y, int Z,
                                       int T) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (e >= n) return;
  const int mu = d >> 1, back = d & 1;
  const int lx = lex[e];
  double re[9], im[9];
  if (lx < 0) {
    for (int k = 0; k < 9; k++) re[k] = im[k] = 0.0;
  } else if (!back) {
    const double2* u = U + ((long)lx * 4 + mu) * 9;
    for (int k = 0; k < 9; k++) {
      re[k] = u[k].x;
      im[k] = u[k].y;
    }
  } else {
    int c[4] = {lx % X, (lx / X) % Y, (lx / (X * Y)) % Z, lx / (X * Y * Z)};
    const int L[4] = {X, Y, Z, T};
    c[mu] = (c[mu] + L[mu] - 1) % L[mu];
    const long nl = c[0] + (long)X * (c[1] + (long)Y * (c[2] + (long)Z * c[3]));
    const double2* u = U + (nl * 4 + mu) * 9;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        re[a * 3 + b] = u[b * 3 + a].x;
        im[a * 3 + b] = -u[b * 3 + a].y;
      }
  }
  store_link9<P>(out, n, e, d, re, im);
}

dwf_status pack_simd_links(dwf_ctx* h, int prec, const int* lex, long n, void* out) {
  dim3 grid((unsigned)((n + 127) / 128), 8), block(128);
  const double2* U = reinterpret_cast<const double2*>(h->links_c128);
  const int* L = h->dims;
  switch (prec) {
    case P64: pack_simd_links_kernel<P64><<<grid, block, 0, h->stream>>>(U, out, lex, n, L[0], L[1], L[2], L[3]); break;
    case P32: pack_simd_links_kernel<P32><<<grid, block, 0, h->stream>>>(U, out, lex, n, L[0], L[1], L[2], L[3]); break;
    case P16: pack_simd_links_kernel<P16><<<grid, block, 0, h->stream>>>(U, out, lex, n, L[0], L[1], L[2], L[3]); break;
    default: pack_simd_links_kernel<PB16><<<grid, block, 0, h->stream>>>(U, out, lex, n, L[0], L[1], L[2], L[3]);
  }
  DWF_CUDA(cudaGetLastError());
  return DWF_OK;
}

size_t simd_link_bytes(int prec, long n) {
  const int nchl = prec == P64 ? 9 : prec == P32 ? 5 : 3;
  return (size_t)8 * nchl * 16 * (size_t)n;
}

}  // namespace

// The sets of block 0 (origin at the lattice origin; every block is a translate of it by a
// multiple of the block shape, which is a symmetry of the periodic lattice):
//   BE, BO: the block's even / odd sites, block-lexicographic order (x fastest);
//   exact operator only: HO = odd sites outside the block next to a BE site (support of
//   Dh_oe of a block vector), HE = even sites outside the block next to a BO or HO site
//   (support of Mpc of a block vector).  Coordinates are taken modulo the lattice, so a block
//   that spans a whole dimension wraps onto itself there and has no halo in it.
dwf_status ensure_simd(dwf_ctx* h, Layout* lay, bool exact, SimdLocal** out) {
  std::unique_ptr<SimdLocal>& slot = lay->simd[exact ? 1 : 0];
  if (slot) {
    *out = slot.get();
    return DWF_OK;
  }
  const Geom& g = lay->g;
  const int* L = g.L;
  const int* B = g.B;
  const long V = g.V;
  auto lexc = [&](const int c[4]) -> long {
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
  };
  auto inblock = [&](const int c[4]) {
    return c[0] < B[0] && c[1] < B[1] && c[2] < B[2] && c[3] < B[3];
  };
  auto step = [&](const int c[4], int d, int n[4]) {
    for (int m = 0; m < 4; m++) n[m] = c[m];
    const int mu = d >> 1;
    n[mu] = (n[mu] + ((d & 1) ? L[mu] - 1 : 1)) % L[mu];
  };
  std::vector<std::array<int, 4>> E, O;
  std::vector<int> idxE(V, -1), idxO(V, -1);
  auto add = [&](std::vector<std::array<int, 4>>& S, std::vector<int>& idx, const int c[4]) {
    const long lx = lexc(c);
    if (idx[lx] >= 0) return;
    idx[lx] = (int)S.size();
    S.push_back({c[0], c[1], c[2], c[3]});
  };
  for (int par = 0; par < 2; par++)
    for (int t = 0; t < B[3]; t++)
      for (int z = 0; z < B[2]; z++)
        for (int y = 0; y < B[1]; y++)
          for (int x = 0; x < B[0]; x++) {
            if (((x + y + z + t) & 1) != par) continue;
            const int c[4] = {x, y, z, t};
            if (par == 0) add(E, idxE, c); else add(O, idxO, c);
          }
  const int nBE = (int)E.size();
  if ((int)O.size() != nBE) return set_error(DWF_ERR_ARG, "block must have even extents");
  if (exact) {
    for (int i = 0; i < nBE; i++)
      for (int d = 0; d < 8; d++) {
        int n[4];
        step(E[i].data(), d, n);
        if (!inblock(n)) add(O, idxO, n);
      }
    for (size_t i = 0; i < O.size(); i++)
      for (int d = 0; d < 8; d++) {
        int n[4];
        step(O[i].data(), d, n);
        if (!inblock(n)) add(E, idxE, n);
      }
  }
  auto S = std::make_unique<SimdLocal>();
  S->exact = exact;
  S->nb = g.nblocks;
  for (int m = 0; m < 4; m++) S->nbk[m] = g.nb[m];
  S->ngroups = (g.nblocks + 31) / 32;
  S->NB = 32 * S->ngroups;
  S->nBE = nBE;
  S->nE = (int)E.size();
  S->nO = (int)O.size();
  S->sB = (long)nBE * S->NB;
  S->sE = (long)S->nE * S->NB;
  S->sO = (long)S->nO * S->NB;
  // neighbour tables
  std::vector<uint32_t> nbrE(8 * (size_t)S->nE, SIMD_ABSENT), nbrO(8 * (size_t)S->nO, SIMD_ABSENT);
  for (int i = 0; i < S->nE; i++)
    for (int d = 0; d < 8; d++) {
      int n[4];
      step(E[i].data(), d, n);
      const int j = idxO[lexc(n)];
      // drop operator: hops that leave the block are absent
      if (j >= 0 && (exact || inblock(n))) nbrE[8 * i + d] = (uint32_t)j;
    }
  for (int i = 0; i < S->nO; i++)
    for (int d = 0; d < 8; d++) {
      int n[4];
      step(O[i].data(), d, n);
      const int j = idxE[lexc(n)];
      if (j >= 0 && (exact || inblock(n))) nbrO[8 * i + d] = (uint32_t)j;
    }
  // schedules: positions by decreasing work (live hops + local term), handed out round robin
  auto sorted = [&](int n, auto cost) {
    std::vector<int> v(n);
    std::iota(v.begin(), v.end(), 0);
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return cost(a) > cost(b); });
    return v;
  };
  auto maskO = [&](int i, bool be_only) {
    uint32_t m = 0;
    for (int d = 0; d < 8; d++) {
      const uint32_t j = nbrO[8 * i + d];
      if (j != SIMD_ABSENT && (!be_only || (int)j < nBE)) m |= 1u << d;
    }
    return m;
  };
  auto maskE = [&](int i) {
    uint32_t m = 0;
    for (int d = 0; d < 8; d++)
      if (nbrE[8 * i + d] != SIMD_ABSENT) m |= 1u << d;
    return m;
  };
  auto pop = [](uint32_t m) { return (int)__builtin_popcount(m); };
  // schedule entries: position | live-hop mask << 24
  if (std::max(S->nE, S->nO) > (int)SIMD_POS_MASK)
    return set_error(DWF_ERR_ARG, "block halo sets too large for the local-solve schedule");
  std::vector<uint32_t> sch;
  auto append = [&](int q, const std::vector<int>& order, auto mask) {
    S->nsch[q] = (int)order.size();
    S->sch_off[q] = (long)sch.size();
    for (int i : order) sch.push_back((uint32_t)i | mask(i) << 24);
  };
  append(0, sorted(S->nO, [&](int i) { return pop(maskO(i, true)); }),
         [&](int i) { return maskO(i, true); });
  append(1, sorted(S->nE, [&](int i) { return pop(maskE(i)) + (i < nBE ? 3 : 0); }), maskE);
  append(2, sorted(S->nO, [&](int i) { return pop(maskO(i, false)); }),
         [&](int i) { return maskO(i, false); });
  append(3, sorted(nBE, [&](int i) { return pop(maskE(i)); }), maskE);
  // element -> site maps: element e = position * NB + block
  auto site_of = [&](const std::array<int, 4>& c, int blk) -> long {
    int bc[4], x[4];
    int b = blk;
    for (int m = 0; m < 4; m++) {
      bc[m] = b % g.nb[m];
      b /= g.nb[m];
    }
    for (int m = 0; m < 4; m++) x[m] = (bc[m] * B[m] + c[m]) % L[m];
    return lexc(x);
  };
  std::vector<int> lexE(S->sE, -1), lexO(S->sO, -1), fwd(S->sB, -1);
  std::vector<int> inv((V / 2 + 31) / 32 * 32, -1);
  for (int i = 0; i < S->nE; i++)
    for (int b = 0; b < S->nb; b++) lexE[(long)i * S->NB + b] = (int)site_of(E[i], b);
  for (int i = 0; i < S->nO; i++)
    for (int b = 0; b < S->nb; b++) lexO[(long)i * S->NB + b] = (int)site_of(O[i], b);
  for (long e = 0; e < S->sB; e++)
    if (lexE[e] >= 0) {
      fwd[e] = lexE[e] / 2;   // whole-lattice even index (x fastest, X even)
      inv[lexE[e] / 2] = (int)e;
    }
  DWF_TRY(upload(nbrE, &S->nbrE));
  DWF_TRY(upload(nbrO, &S->nbrO));
  DWF_TRY(upload(sch, &S->sch));
  DWF_TRY(upload(lexE, &S->lexE));
  DWF_TRY(upload(lexO, &S->lexO));
  DWF_TRY(upload(fwd, &S->fwd));
  DWF_TRY(upload(inv, &S->inv));
  slot = std::move(S);
  *out = slot.get();
  return DWF_OK;
}

static dwf_status ensure_simd_links(dwf_ctx* h, SimdLocal* S, int prec) {
  if (S->links_valid[prec]) return DWF_OK;
  if (!S->linksE[prec]) DWF_CUDA(cudaMalloc(&S->linksE[prec], simd_link_bytes(prec, S->sE)));
  if (!S->linksO[prec]) DWF_CUDA(cudaMalloc(&S->linksO[prec], simd_link_bytes(prec, S->sO)));
  DWF_TRY(pack_simd_links(h, prec, S->lexE, S->sE, S->linksE[prec]));
  DWF_TRY(pack_simd_links(h, prec, S->lexO, S->sO, S->linksO[prec]));
  S->links_valid[prec] = true;
  return DWF_OK;
}

static cudaError_t simd_launch(int prec, const SimdArgs& a, int Ls, int v, int* cap, int nsm,
                               cudaStream_t st, bool query) {
  switch (prec) {
    case P64: return simd_launch_p<P64>(a, Ls, v, cap, nsm, st, query);
    case P32: return simd_launch_p<P32>(a, Ls, v, cap, nsm, st, query);
    case P16: return simd_launch_p<P16>(a, Ls, v, cap, nsm, st, query);
    default: return simd_launch_p<PB16>(a, Ls, v, cap, nsm, st, query);
  }
}

// Launch-variant tuner of the local-solve kernel (FP32/FP16/BF16 have three variants: ring
// depth and register budget): the first calls per precision run every variant once untimed,
// then twice timed with CUDA events on the stream; once all events have completed (checked
// without blocking at later calls) the fastest is kept.  Calls under stream capture use the
// current choice.  DWF_LOCAL_VARIANT=<v> forces variant v.
constexpr int SIMD_NV = 3, SIMD_TUNE_ROUNDS = 4;

bool simd_variant_decided(const SimdLocal* S, int prec) {
  if (prec == P64) return true;
  if (const char* f = getenv("DWF_LOCAL_VARIANT")) {
    const int v = atoi(f);
    if (v >= 0 && v < SIMD_NV) return true;
  }
  return S->tune_chosen[prec] >= 0;
}

static int simd_pick(SimdLocal* S, int prec, cudaStream_t st, bool capturing, int* timed) {
  *timed = -1;
  if (prec == P64) return 0;
  if (const char* f = getenv("DWF_LOCAL_VARIANT")) {
    const int v = atoi(f);
    if (v >= 0 && v < SIMD_NV) return v;
  }
  int& chosen = S->tune_chosen[prec];
  int& next = S->tune_next[prec];
  const int nt = SIMD_TUNE_ROUNDS * SIMD_NV;
  if (chosen >= 0) return chosen;
  if (next >= SIMD_NV + nt) {   // every candidate timed: decide once the events are done
    if (capturing) return 0;
    bool done = true;
    for (int i = 0; i < 2 * nt; i++)
      done = done && cudaEventQuery(S->tune_ev[prec][i]) == cudaSuccess;
    cudaGetLastError();
    if (!done) return 0;
    float best = 0.f, tv[SIMD_NV];
    for (int v = 0; v < SIMD_NV; v++) {
      float t = 0.f;
      for (int i = v; i < nt; i += SIMD_NV) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S->tune_ev[prec][2 * i], S->tune_ev[prec][2 * i + 1]);
        t += ms;
      }
      tv[v] = t / SIMD_TUNE_ROUNDS;
      if (chosen < 0 || t < best) {
        best = t;
        chosen = v;
      }
    }
    if (getenv("DWF_TUNE_LOG"))
      fprintf(stderr, "dwf tune local solve P%d: variant %d (%.3f / %.3f / %.3f ms)\n", prec,
              chosen, tv[0], tv[1], tv[2]);
    for (auto& e : S->tune_ev[prec]) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    return chosen;
  }
  if (capturing) return 0;
  if (next == 0)
    for (int i = 0; i < 2 * nt; i++) cudaEventCreate(&S->tune_ev[prec][i]);
  const int v = next % SIMD_NV;
  if (next >= SIMD_NV) *timed = next - SIMD_NV;
  next++;
  return v;
}

dwf_status simd_local_solve(dwf_ctx* h, SimdLocal* S, int prec, int l, const void* r_outer,
                            int prec_outer, long Vp_outer, double num, const double* den,
                            const SimdFields& F, int ncol, int col) {
  DWF_TRY(ensure_simd_links(h, S, prec));
  SimdArgs a{};
  a.ncol = ncol;
  a.col = col;
  for (int m = 0; m < 4; m++) a.nbk[m] = S->nbk[m];
  a.NB = S->NB;
  a.nb = S->nb;
  a.nBE = S->nBE;
  a.nE = S->nE;
  a.nO = S->nO;
  a.ngroups = S->ngroups;
  a.sB = S->sB;
  a.sE = S->sE;
  a.sO = S->sO;
  a.nbrE = S->nbrE;
  a.nbrO = S->nbrO;
  for (int q = 0; q < 4; q++) {
    a.sch[q] = S->sch + S->sch_off[q];
    a.nsch[q] = S->nsch[q];
  }
  a.linksE = S->linksE[prec];
  a.linksO = S->linksO[prec];
  a.fwd = S->fwd;
  a.x = F.x;
  a.p = F.p;
  a.u = F.u;
  a.r = F.r;
  a.t = F.t;
  a.y = F.y;
  a.r_outer = r_outer;
  a.prec_outer = prec_outer;
  a.Vp_outer = Vp_outer;
  a.num = num;
  a.den = den;
  const Matrices& M = h->mats;
  const bool trivial = M.dplus_trivial;
  const double pre = trivial ? h->b : 1.0;
  a.k64 = make_coef5<double>(M.m5_alpha, M.m5_beta, h->mf, h->b, h->c, pre, h->Ls);
  a.k32 = make_coef5<float>(M.m5_alpha, M.m5_beta, h->mf, h->b, h->c, pre, h->Ls);
  a.hs_b = trivial ? -0.25 * h->b : -0.25;
  a.trivial = trivial ? 1 : 0;
  a.l = l;
  a.wait_ns = h->wait_ns;
  a.err = h->dev_err;
  // grid: every CTA resident (cooperative launch); C CTAs per slot of 32-block groups
  int dev = 0, nsm = 1, cap = 0;
  DWF_CUDA(cudaGetDevice(&dev));
  DWF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(h->stream, &capst);
  int timed = -1;
  const int v = simd_pick(S, prec, h->stream, capst != cudaStreamCaptureStatusNone, &timed);
  DWF_CUDA(simd_launch(prec, a, h->Ls, v, &cap, nsm, h->stream, true));
  if (cap < 1) return set_error(DWF_ERR_CUDA, "local-solve kernel cannot be resident");
  const int most = std::max(1, std::max(S->nE, S->nO) / 2);   // positions per CTA >= 2
  int C = std::max(1, std::min(cap / S->ngroups, most));
  const int nslots = std::max(1, std::min(S->ngroups, cap / C));
  a.C = C;
  a.nslots = nslots;
  if (S->cap_slots < nslots || S->cap_C < C) {
    cudaFree(S->ctr);
    cudaFree(S->partial);
    S->ctr = nullptr;
    S->partial = nullptr;
    DWF_CUDA(cudaMalloc(&S->ctr, nslots * sizeof(unsigned)));
    DWF_CUDA(cudaMalloc(&S->partial, (size_t)nslots * C * 32 * sizeof(double)));
    S->cap_slots = nslots;
    S->cap_C = C;
  }
  a.ctr = S->ctr;
  a.partial = S->partial;
  DWF_CUDA(cudaMemsetAsync(S->ctr, 0, nslots * sizeof(unsigned), h->stream));
  const double R = (double)real_bytes(prec);
  // algorithmic bytes per local iteration: the four hop stages read their input once and
  // write their output once per site and slice, read the links of their sites once, plus the
  // local terms and the CG vectors
  const double per = 24.0 * R * h->Ls;
  const double nbk = (double)S->nb;
  const double links = 144.0 * R;
  const double it_bytes =
      nbk * ((S->nBE + S->nO) * per + (double)S->nO * links +          // P1
             (S->nBE + S->nE) * per + 2.0 * S->nBE * per + S->nE * links +   // P2
             (S->nE + S->nO) * per + (double)S->nO * links +            // P3
             (S->nO + 4.0 * S->nBE) * per + S->nBE * links +            // P4
             6.0 * S->nBE * per);                                        // P5
  ProfScope ps(&h->prof, h->stream, prec == P16 ? "local_solve_f16"
                                   : prec == PB16 ? "local_solve_bf16"
                                   : prec == P32 ? "local_solve_f32" : "local_solve_f64",
               it_bytes * l, 0.0);
  if (timed >= 0) DWF_CUDA(cudaEventRecord(S->tune_ev[prec][2 * timed], h->stream));
  DWF_CUDA(simd_launch(prec, a, h->Ls, v, &cap, nsm, h->stream, false));
  if (timed >= 0) DWF_CUDA(cudaEventRecord(S->tune_ev[prec][2 * timed + 1], h->stream));
  return DWF_OK;
}

}  // namespace dwf
