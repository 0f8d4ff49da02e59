// Site orderings, neighbour tables, link packing and caller <-> internal field conversion.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <unordered_map>

#include "dwf_internal.h"

namespace dwf {

Layout::~Layout() {
  for (int p = 0; p < 2; p++) {
    cudaFree(nbr[p]);
    cudaFree(lex[p]);
    for (int q = 0; q < 4; q++) cudaFree(links[q][p]);
  }
  cudaFree(cb_even);
  cudaFree(cb_inv);
}

// Coordinates (x, y, z, t) of internal site idx of parity p; false for padding.
static bool coords_of(const Geom& g, int p, long idx, int c[4]) {
  const long blk = idx / g.Vhb_pad;
  const long j = idx % g.Vhb_pad;
  if (j >= g.Vhb) return false;
  long b = blk;
  int bc[4];
  for (int m = 0; m < 4; m++) {
    bc[m] = (int)(b % g.nb[m]);
    b /= g.nb[m];
  }
  const int hx = g.B[0] / 2;
  long r = j;
  const int jx = (int)(r % hx);
  r /= hx;
  const int ly = (int)(r % g.B[1]);
  r /= g.B[1];
  const int lz = (int)(r % g.B[2]);
  const int lt = (int)(r / g.B[2]);
  c[1] = bc[1] * g.B[1] + ly;
  c[2] = bc[2] * g.B[2] + lz;
  c[3] = bc[3] * g.B[3] + lt;
  const int x0 = bc[0] * g.B[0] + 2 * jx;
  c[0] = x0 + ((p + c[1] + c[2] + c[3]) & 1);
  return true;
}

static long index_of(const Geom& g, const int c[4], int* blk_out) {
  int bc[4], l[4];
  for (int m = 0; m < 4; m++) {
    bc[m] = c[m] / g.B[m];
    l[m] = c[m] % g.B[m];
  }
  const long blk = bc[0] + (long)g.nb[0] * (bc[1] + (long)g.nb[1] * (bc[2] + (long)g.nb[2] * bc[3]));
  const long j = l[0] / 2 + (long)(g.B[0] / 2) * (l[1] + (long)g.B[1] * (l[2] + (long)g.B[2] * l[3]));
  if (blk_out) *blk_out = (int)blk;
  return blk * g.Vhb_pad + j;
}

dwf_status get_layout(dwf_ctx* h, const int block[4], Layout** out) {
  for (auto& l : h->layouts)
    if (l->g.same(block)) {
      *out = l.get();
      return DWF_OK;
    }
  for (int m = 0; m < 4; m++) {
    if (block[m] < 2 || block[m] % 2 != 0 || h->dims[m] % block[m] != 0)
      return set_error(DWF_ERR_ARG, "block dims must be even and divide the lattice dims");
  }
  auto lay = std::make_unique<Layout>();
  Geom& g = lay->g;
  g.V = 1;
  g.nblocks = 1;
  for (int m = 0; m < 4; m++) {
    g.L[m] = h->dims[m];
    g.B[m] = block[m];
    g.nb[m] = h->dims[m] / block[m];
    g.nblocks *= g.nb[m];
    g.V *= h->dims[m];
  }
  g.Vhb = block[0] * block[1] * block[2] * block[3] / 2;
  g.Vhb_pad = (g.Vhb + 31) / 32 * 32;
  g.Vp = (long)g.nblocks * g.Vhb_pad;
  g.Ls = h->Ls;

  std::vector<uint32_t> nbr(8 * (size_t)g.Vp);
  std::vector<int> lex(g.Vp), cbe(g.Vp);
  const int X = g.L[0], Y = g.L[1], Z = g.L[2];
  for (int p = 0; p < 2; p++) {
    for (long idx = 0; idx < g.Vp; idx++) {
      int c[4];
      if (!coords_of(g, p, idx, c)) {
        lex[idx] = -1;
        if (p == 0) cbe[idx] = -1;
        for (int d = 0; d < 8; d++) nbr[d * g.Vp + idx] = 0u;
        continue;
      }
      const long lx = c[0] + (long)X * (c[1] + (long)Y * (c[2] + (long)Z * c[3]));
      lex[idx] = (int)lx;
      if (p == 0) cbe[idx] = (int)(lx / 2);
      int myblk;
      index_of(g, c, &myblk);
      for (int mu = 0; mu < 4; mu++) {
        for (int back = 0; back < 2; back++) {
          int n[4] = {c[0], c[1], c[2], c[3]};
          n[mu] = (n[mu] + (back ? g.L[mu] - 1 : 1)) % g.L[mu];
          int nblk;
          const long nidx = index_of(g, n, &nblk);
          nbr[(2 * mu + back) * g.Vp + idx] = (uint32_t)nidx | (nblk != myblk ? NBR_FACE : 0u);
        }
      }
    }
    DWF_CUDA(cudaMalloc(&lay->nbr[p], nbr.size() * sizeof(uint32_t)));
    DWF_CUDA(cudaMalloc(&lay->lex[p], lex.size() * sizeof(int)));
    DWF_CUDA(cudaMemcpy(lay->nbr[p], nbr.data(), nbr.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice));
    DWF_CUDA(cudaMemcpy(lay->lex[p], lex.data(), lex.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
  }
  DWF_CUDA(cudaMalloc(&lay->cb_even, cbe.size() * sizeof(int)));
  DWF_CUDA(cudaMemcpy(lay->cb_even, cbe.data(), cbe.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  std::vector<int> inv((g.V / 2 + 31) / 32 * 32, -1);
  for (long idx = 0; idx < g.Vp; idx++)
    if (cbe[idx] >= 0) inv[cbe[idx]] = (int)idx;
  DWF_CUDA(cudaMalloc(&lay->cb_inv, inv.size() * sizeof(int)));
  DWF_CUDA(cudaMemcpy(lay->cb_inv, inv.data(), inv.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
  *out = lay.get();
  h->layouts.push_back(std::move(lay));
  return DWF_OK;
}

// ---------------------------------------------------------------------------------------
// Halo tables of the exact block operator.
// ---------------------------------------------------------------------------------------
Halo::~Halo() {
  cudaFree(nbr_be);
  cudaFree(nbr_bo);
  cudaFree(nbr_ho);
  cudaFree(nbr_he);
  cudaFree(ls_ho);
  cudaFree(ls_he);
  for (int p = 0; p < 4; p++) {
    cudaFree(links_ho[p]);
    cudaFree(links_he[p]);
  }
}

static long lex_of(const Geom& g, const int c[4]) {
  return c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
}

static void coords_lex(const Geom& g, long lx, int c[4]) {
  for (int m = 0; m < 4; m++) {
    c[m] = (int)(lx % g.L[m]);
    lx /= g.L[m];
  }
}

static void neighbour(const Geom& g, const int c[4], int d, int n[4]) {
  for (int m = 0; m < 4; m++) n[m] = c[m];
  const int mu = d >> 1;
  n[mu] = (n[mu] + ((d & 1) ? g.L[mu] - 1 : 1)) % g.L[mu];
}

template <typename T>
static dwf_status upload_vec(const std::vector<T>& v, T** dst) {
  DWF_CUDA(cudaMalloc(dst, v.size() * sizeof(T)));
  DWF_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DWF_OK;
}

dwf_status ensure_halo(dwf_ctx* h, Layout* lay) {
  (void)h;
  if (lay->halo) return DWF_OK;
  const Geom& g = lay->g;
  const int nb = g.nblocks;
  std::vector<std::vector<long>> ho(nb), he(nb);   // sorted lexicographic indices
  auto blk_of = [&](const int c[4]) {
    int b;
    index_of(g, c, &b);
    return b;
  };
  for (int b = 0; b < nb; b++) {
    std::vector<long>& O = ho[b];
    for (long j = 0; j < g.Vhb; j++) {
      int c[4];
      coords_of(g, 0, (long)b * g.Vhb_pad + j, c);
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        if (blk_of(n) != b) O.push_back(lex_of(g, n));
      }
    }
    std::sort(O.begin(), O.end());
    O.erase(std::unique(O.begin(), O.end()), O.end());
    std::vector<long>& E = he[b];
    auto add_even = [&](const int c[4]) {
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        if (blk_of(n) != b) E.push_back(lex_of(g, n));
      }
    };
    for (long j = 0; j < g.Vhb; j++) {
      int c[4];
      coords_of(g, 1, (long)b * g.Vhb_pad + j, c);
      add_even(c);
    }
    for (long lx : O) {
      int c[4];
      coords_lex(g, lx, c);
      add_even(c);
    }
    std::sort(E.begin(), E.end());
    E.erase(std::unique(E.begin(), E.end()), E.end());
  }
  auto H = std::make_unique<Halo>();
  for (int b = 0; b < nb; b++) {
    H->Ho_b = std::max(H->Ho_b, (int)ho[b].size());
    H->He_b = std::max(H->He_b, (int)he[b].size());
  }
  H->Ho_pad = std::max(32, (H->Ho_b + 31) / 32 * 32);
  H->He_pad = std::max(32, (H->He_b + 31) / 32 * 32);
  H->Ho_tot = (long)nb * H->Ho_pad;
  H->He_tot = (long)nb * H->He_pad;
  // Order each block's halo lists by the set of neighbours that exist (an 8-bit mask), so a
  // warp's 32 halo sites take the same hop directions (no divergence over absent hops).
  {
    auto in_set = [](const std::vector<long>& v, long x) {
      return std::binary_search(v.begin(), v.end(), x);
    };
    for (int b = 0; b < nb; b++) {
      for (int odd = 0; odd < 2; odd++) {
        std::vector<long>& L = odd ? ho[b] : he[b];
        const std::vector<long>& other = odd ? he[b] : ho[b];
        std::vector<std::pair<int, long>> keyed;
        keyed.reserve(L.size());
        for (long lx : L) {
          int c[4], mask = 0;
          coords_lex(g, lx, c);
          for (int d = 0; d < 8; d++) {
            int n[4];
            neighbour(g, c, d, n);
            if (blk_of(n) == b || in_set(other, lex_of(g, n))) mask |= 1 << d;
          }
          keyed.push_back({mask, lx});
        }
        std::sort(keyed.begin(), keyed.end());
        for (size_t k = 0; k < keyed.size(); k++) L[k] = keyed[k].second;
      }
    }
  }
  // position of a site in a (reordered) halo list
  std::vector<std::unordered_map<long, long>> hpos_o(nb), hpos_e(nb);
  for (int b = 0; b < nb; b++) {
    for (size_t k = 0; k < ho[b].size(); k++) hpos_o[b][ho[b][k]] = (long)k;
    for (size_t k = 0; k < he[b].size(); k++) hpos_e[b][he[b][k]] = (long)k;
  }
  std::vector<uint32_t> be(8 * (size_t)g.Vp, NBR_FACE), bo(8 * (size_t)g.Vp, NBR_FACE);
  std::vector<uint32_t> nho(8 * (size_t)H->Ho_tot, NBR_FACE), nhe(8 * (size_t)H->He_tot, NBR_FACE);
  std::vector<int> lho(H->Ho_tot, 0), lhe(H->He_tot, 0);
  // entry for a neighbour n of a site of block b: in block -> its index in the other
  // parity; in the halo list `hl` -> NBR_HALO | b * hpad + position; else absent.
  auto entry = [&](int b, const int n[4], bool to_odd_halo, int hpad) -> uint32_t {
    int nbk;
    const long nidx = index_of(g, n, &nbk);
    if (nbk == b) return (uint32_t)nidx;
    const auto& m = to_odd_halo ? hpos_o[b] : hpos_e[b];
    const auto it = m.find(lex_of(g, n));
    if (it == m.end()) return NBR_FACE;
    return NBR_HALO | (uint32_t)((long)b * hpad + it->second);
  };
  for (int b = 0; b < nb; b++) {
    for (long j = 0; j < g.Vhb; j++) {
      const long idx = (long)b * g.Vhb_pad + j;
      int c[4];
      coords_of(g, 0, idx, c);
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        be[d * g.Vp + idx] = entry(b, n, true, H->Ho_pad);
      }
      coords_of(g, 1, idx, c);
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        bo[d * g.Vp + idx] = entry(b, n, false, H->He_pad);
      }
    }
    for (size_t k = 0; k < ho[b].size(); k++) {
      const long i = (long)b * H->Ho_pad + (long)k;
      int c[4];
      coords_lex(g, ho[b][k], c);
      lho[i] = (int)index_of(g, c, nullptr);
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        nho[d * H->Ho_tot + i] = entry(b, n, false, H->He_pad);
      }
    }
    for (size_t k = 0; k < he[b].size(); k++) {
      const long i = (long)b * H->He_pad + (long)k;
      int c[4];
      coords_lex(g, he[b][k], c);
      lhe[i] = (int)index_of(g, c, nullptr);
      for (int d = 0; d < 8; d++) {
        int n[4];
        neighbour(g, c, d, n);
        nhe[d * H->He_tot + i] = entry(b, n, true, H->Ho_pad);
      }
    }
  }
  DWF_TRY(upload_vec(be, &H->nbr_be));
  DWF_TRY(upload_vec(bo, &H->nbr_bo));
  DWF_TRY(upload_vec(nho, &H->nbr_ho));
  DWF_TRY(upload_vec(nhe, &H->nbr_he));
  DWF_TRY(upload_vec(lho, &H->ls_ho));
  DWF_TRY(upload_vec(lhe, &H->ls_he));
  lay->halo = std::move(H);
  // links packed before the halo existed: repack so the halo copies get gathered
  for (int p = 0; p < 4; p++) lay->links_valid[p] = false;
  return DWF_OK;
}

// ---------------------------------------------------------------------------------------
// Links.
// ---------------------------------------------------------------------------------------
template <int P>
__global__ void pack_links_kernel(const double2* __restrict__ U, void* out,
                                  const uint32_t* __restrict__ nbr, const int* __restrict__ lexp,
                                  const int* __restrict__ lexq, long Vp) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (idx >= Vp) return;
  const int mu = d >> 1, back = d & 1;
  const int lx = lexp[idx];
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
    const int nl = lexq[nbr[(long)d * Vp + idx] & NBR_IDX];
    const double2* u = U + ((long)nl * 4 + mu) * 9;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        re[a * 3 + b] = u[b * 3 + a].x;
        im[a * 3 + b] = -u[b * 3 + a].y;
      }
  }
  store_link9<P>(out, Vp, idx, d, re, im);
}

// Copies the links of the sites listed in `site` ([n]) into a contiguous [8][NCHL][n] array.
template <int P>
__global__ void gather_links_kernel(const uint4* __restrict__ src, long Vp, uint4* dst, long n,
                                    const int* __restrict__ site) {
  constexpr int NCHL = Prec<P>::NCHL;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (i >= n) return;
  const long g = site[i];
  for (int k = 0; k < NCHL; k++)
    dst[((long)d * NCHL + k) * n + i] = src[((long)d * NCHL + k) * Vp + g];
}

static size_t link_bytes(int prec, long Vp) {
  const int nchl = prec == P64 ? 9 : prec == P32 ? 5 : 3;
  return (size_t)8 * nchl * 16 * (size_t)Vp;
}

dwf_status ensure_links(dwf_ctx* h, Layout* lay, int prec) {
  if (lay->links_valid[prec]) return DWF_OK;
  const Geom& g = lay->g;
  for (int p = 0; p < 2; p++) {
    if (!lay->links[prec][p]) {
      cudaError_t e = cudaMalloc(&lay->links[prec][p], link_bytes(prec, g.Vp));
      if (e != cudaSuccess) return set_error(DWF_ERR_NOMEM, "links allocation failed");
    }
    dim3 grid((unsigned)((g.Vp + 127) / 128), 8), block(128);
    const double2* U = reinterpret_cast<const double2*>(h->links_c128);
    void* out = lay->links[prec][p];
    switch (prec) {
      case P64: pack_links_kernel<P64><<<grid, block, 0, h->stream>>>(U, out, lay->nbr[p], lay->lex[p], lay->lex[1 - p], g.Vp); break;
      case P32: pack_links_kernel<P32><<<grid, block, 0, h->stream>>>(U, out, lay->nbr[p], lay->lex[p], lay->lex[1 - p], g.Vp); break;
      case P16: pack_links_kernel<P16><<<grid, block, 0, h->stream>>>(U, out, lay->nbr[p], lay->lex[p], lay->lex[1 - p], g.Vp); break;
      default: pack_links_kernel<PB16><<<grid, block, 0, h->stream>>>(U, out, lay->nbr[p], lay->lex[p], lay->lex[1 - p], g.Vp);
    }
    DWF_CUDA(cudaGetLastError());
  }
  // the block halos keep their own contiguous copies of the links of their sites
  if (lay->halo) {
    Halo& H = *lay->halo;
    for (int odd = 0; odd < 2; odd++) {
      const long n = odd ? H.Ho_tot : H.He_tot;
      void*& dst = odd ? H.links_ho[prec] : H.links_he[prec];
      if (!dst) DWF_CUDA(cudaMalloc(&dst, link_bytes(prec, n)));
      dim3 grid((unsigned)((n + 127) / 128), 8), block(128);
      const uint4* src = reinterpret_cast<const uint4*>(lay->links[prec][odd]);
      const int* site = odd ? H.ls_ho : H.ls_he;
      switch (prec) {
        case P64: gather_links_kernel<P64><<<grid, block, 0, h->stream>>>(src, g.Vp, (uint4*)dst, n, site); break;
        case P32: gather_links_kernel<P32><<<grid, block, 0, h->stream>>>(src, g.Vp, (uint4*)dst, n, site); break;
        case P16: gather_links_kernel<P16><<<grid, block, 0, h->stream>>>(src, g.Vp, (uint4*)dst, n, site); break;
        default: gather_links_kernel<PB16><<<grid, block, 0, h->stream>>>(src, g.Vp, (uint4*)dst, n, site);
      }
      DWF_CUDA(cudaGetLastError());
    }
  }
  lay->links_valid[prec] = true;
  return DWF_OK;
}

// ---------------------------------------------------------------------------------------
// Fields: caller complex128 <-> internal chunked layout.
// ---------------------------------------------------------------------------------------
template <int P>
__global__ void pack_field_kernel(const double2* __restrict__ src, void* dst,
                                  const int* __restrict__ map, long Vp, long nsrc, double scale,
                                  int div2) {
  using A = typename Prec<P>::acc;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (idx >= Vp) return;
  int m = map[idx];
  Spinor<A> v;
  if (m < 0) {
    zero(v);
  } else {
    if (div2) m >>= 1;
    const double2* q = src + ((long)s * nsrc + m) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) v.c[k] = {A(q[k].x * scale), A(q[k].y * scale)};
  }
  store_spinor<P>(dst, Vp, idx, s, v);
}

template <int P>
__global__ void unpack_field_kernel(const void* src, double2* __restrict__ dst,
                                    const int* __restrict__ map, long Vp, long ndst,
                                    double inv_scale, int div2) {
  using A = typename Prec<P>::acc;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (idx >= Vp) return;
  int m = map[idx];
  if (m < 0) return;
  if (div2) m >>= 1;
  Spinor<A> v;
  load_spinor<P>(v, src, Vp, idx, s);
  double2* q = dst + ((long)s * ndst + m) * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) q[k] = make_double2((double)v.c[k].x * inv_scale,
                                                   (double)v.c[k].y * inv_scale);
}

static dwf_status launch_pack(dwf_ctx* h, const Geom& g, const void* src, void* dst,
                              const int* map, long nsrc, double scale, int div2, int prec) {
  dim3 grid((unsigned)((g.Vp + 127) / 128), g.Ls), block(128);
  const double2* s = reinterpret_cast<const double2*>(src);
  switch (prec) {
    case P64: pack_field_kernel<P64><<<grid, block, 0, h->stream>>>(s, dst, map, g.Vp, nsrc, scale, div2); break;
    case P32: pack_field_kernel<P32><<<grid, block, 0, h->stream>>>(s, dst, map, g.Vp, nsrc, scale, div2); break;
    case P16: pack_field_kernel<P16><<<grid, block, 0, h->stream>>>(s, dst, map, g.Vp, nsrc, scale, div2); break;
    default: pack_field_kernel<PB16><<<grid, block, 0, h->stream>>>(s, dst, map, g.Vp, nsrc, scale, div2);
  }
  DWF_CUDA(cudaGetLastError());
  return DWF_OK;
}

static dwf_status launch_unpack(dwf_ctx* h, const Geom& g, const void* src, void* dst,
                                const int* map, long ndst, double scale, int div2, int prec) {
  dim3 grid((unsigned)((g.Vp + 127) / 128), g.Ls), block(128);
  double2* d = reinterpret_cast<double2*>(dst);
  const double inv = 1.0 / scale;
  switch (prec) {
    case P64: unpack_field_kernel<P64><<<grid, block, 0, h->stream>>>(src, d, map, g.Vp, ndst, inv, div2); break;
    case P32: unpack_field_kernel<P32><<<grid, block, 0, h->stream>>>(src, d, map, g.Vp, ndst, inv, div2); break;
    case P16: unpack_field_kernel<P16><<<grid, block, 0, h->stream>>>(src, d, map, g.Vp, ndst, inv, div2); break;
    default: unpack_field_kernel<PB16><<<grid, block, 0, h->stream>>>(src, d, map, g.Vp, ndst, inv, div2);
  }
  DWF_CUDA(cudaGetLastError());
  return DWF_OK;
}

dwf_status pack_even(dwf_ctx* h, Layout* lay, const void* src_c128, void* dst, int prec,
                     double scale) {
  return launch_pack(h, lay->g, src_c128, dst, lay->cb_even, lay->g.V / 2, scale, 0, prec);
}

dwf_status unpack_even(dwf_ctx* h, Layout* lay, const void* src, int prec, void* dst_c128,
                       double scale) {
  return launch_unpack(h, lay->g, src, dst_c128, lay->cb_even, lay->g.V / 2, scale, 0, prec);
}

dwf_status pack_full(dwf_ctx* h, Layout* lay, const void* src_c128, void* dst_even,
                     void* dst_odd, int prec) {
  DWF_TRY(launch_pack(h, lay->g, src_c128, dst_even, lay->lex[0], lay->g.V, 1.0, 0, prec));
  return launch_pack(h, lay->g, src_c128, dst_odd, lay->lex[1], lay->g.V, 1.0, 0, prec);
}

dwf_status unpack_full(dwf_ctx* h, Layout* lay, const void* src_even, const void* src_odd,
                       int prec, void* dst_c128) {
  DWF_TRY(launch_unpack(h, lay->g, src_even, dst_c128, lay->lex[0], lay->g.V, 1.0, 0, prec));
  return launch_unpack(h, lay->g, src_odd, dst_c128, lay->lex[1], lay->g.V, 1.0, 0, prec);
}

// ---------------------------------------------------------------------------------------
// Fifth-dimension matrices (host, double), uploaded in double and float.
// ---------------------------------------------------------------------------------------
static std::vector<double> kmat(int Ls, double mf, int chi) {
  // chi 0 (P+ rows): K psi_s = psi_{s-1}; chi 1 (P- rows): K psi_s = psi_{s+1}
  std::vector<double> k(Ls * Ls, 0.0);
  for (int s = 0; s < Ls; s++) {
    if (chi == 0) {
      if (s > 0) k[s * Ls + s - 1] = 1.0; else k[s * Ls + Ls - 1] = -mf;
    } else {
      if (s + 1 < Ls) k[s * Ls + s + 1] = 1.0; else k[s * Ls] = -mf;
    }
  }
  return k;
}

static bool invert(std::vector<double> a, int n, std::vector<double>& inv) {
  inv.assign(n * n, 0.0);
  for (int i = 0; i < n; i++) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (a[piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; k++) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    const double d = a[c * n + c];
    for (int k = 0; k < n; k++) {
      a[c * n + k] /= d;
      inv[c * n + k] /= d;
    }
    for (int r = 0; r < n; r++) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; k++) {
        a[r * n + k] -= f * a[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  return true;
}

static std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b,
                                  int n) {
  std::vector<double> c(n * n, 0.0);
  for (int i = 0; i < n; i++)
    for (int k = 0; k < n; k++)
      for (int j = 0; j < n; j++) c[i * n + j] += a[i * n + k] * b[k * n + j];
  return c;
}

static std::vector<double> transpose(const std::vector<double>& a, int n) {
  std::vector<double> t(n * n);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) t[j * n + i] = a[i * n + j];
  return t;
}

static dwf_status upload(const std::vector<double>& m, void* dst[2]) {
  const size_t n = m.size();
  if (!dst[0]) DWF_CUDA(cudaMalloc(&dst[0], n * sizeof(double)));
  if (!dst[1]) DWF_CUDA(cudaMalloc(&dst[1], n * sizeof(float)));
  std::vector<float> f(m.begin(), m.end());
  DWF_CUDA(cudaMemcpy(dst[0], m.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  DWF_CUDA(cudaMemcpy(dst[1], f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  return DWF_OK;
}

dwf_status build_matrices(dwf_ctx* h) {
  const int Ls = h->Ls;
  Matrices& M = h->mats;
  const double a = (4.0 - h->M5) * h->b + 1.0;   // M5op = a + beta K
  const double be = (4.0 - h->M5) * h->c - 1.0;
  M.m5_alpha = a;
  M.m5_beta = be;
  M.dplus_trivial = (h->c == 0.0);
  std::vector<double> dp, dpt, dpm5i, m5idpt;
  for (int chi = 0; chi < 2; chi++) {
    std::vector<double> K = kmat(Ls, h->mf, chi), D(Ls * Ls), M5(Ls * Ls);
    for (int i = 0; i < Ls * Ls; i++) {
      const double id = (i % (Ls + 1) == 0) ? 1.0 : 0.0;
      D[i] = h->b * id + h->c * K[i];
      M5[i] = a * id + be * K[i];
    }
    std::vector<double> M5i;
    if (!invert(M5, Ls, M5i)) return set_error(DWF_ERR_ARG, "M5op is singular");
    std::vector<double> DM = matmul(D, M5i, Ls);
    // the post matrix of stage A absorbs the pre-op factor b when D+ = b
    if (M.dplus_trivial)
      for (auto& v : DM) v *= h->b;
    std::vector<double> MDt = matmul(transpose(M5i, Ls), transpose(D, Ls), Ls);
    dp.insert(dp.end(), D.begin(), D.end());
    std::vector<double> Dt = transpose(D, Ls);
    dpt.insert(dpt.end(), Dt.begin(), Dt.end());
    dpm5i.insert(dpm5i.end(), DM.begin(), DM.end());
    m5idpt.insert(m5idpt.end(), MDt.begin(), MDt.end());
  }
  M.dp = dp;
  M.dpt = dpt;
  M.dpm5i = dpm5i;
  M.m5idpt = m5idpt;
  DWF_TRY(upload(dp, M.d_dp));
  DWF_TRY(upload(dpt, M.d_dpt));
  DWF_TRY(upload(dpm5i, M.d_dpm5i));
  DWF_TRY(upload(m5idpt, M.d_m5idpt));
  // tensor-core operands: B[k][n] = M[n][k] stored K-major (row n, column k) in 8x8 core
  // matrices, zero padded to 16 x 16, FP16
  const std::vector<double>* src[3] = {&dpm5i, &m5idpt, &dpt};
  for (int w = 0; w < 3; w++) {
    std::vector<__half> hb(2 * 256, __float2half(0.f));
    for (int chi = 0; chi < 2; chi++)
      for (int n = 0; n < Ls; n++)
        for (int k = 0; k < Ls; k++) {
          const int off = (n / 8) * 128 + (k / 8) * 64 + (n % 8) * 8 + (k % 8);
          hb[chi * 256 + off] = __float2half((float)(*src[w])[(chi * Ls + n) * Ls + k]);
        }
    if (!M.d_post_h[w]) DWF_CUDA(cudaMalloc(&M.d_post_h[w], hb.size() * sizeof(__half)));
    DWF_CUDA(cudaMemcpy(M.d_post_h[w], hb.data(), hb.size() * sizeof(__half),
                        cudaMemcpyHostToDevice));
  }
  const char* e = getenv("DWF_DISABLE_TC");
  M.use_tc = !(e && e[0] == '1');
  const char* pm = getenv("DWF_POST");   // auto | matrix | recurrence
  M.post_mode = !pm ? 0 : pm[0] == 'm' ? 1 : pm[0] == 'r' ? 2 : 0;
  if (!M.use_tc && M.post_mode == 0) M.post_mode = 1;
  M.struct_ok = std::fabs(be) < std::fabs(a);
  return DWF_OK;
}

}  // namespace dwf

// ---------------------------------------------------------------------------------------
// Launchers on caller-provided memory (used by the allocation-free entry point).
// ---------------------------------------------------------------------------------------
namespace dwf {

cudaError_t launch_pack_links_to(int prec, const void* U, void* out, const uint32_t* nbr,
                                 const int* lexp, const int* lexq, long Vp, cudaStream_t st) {
  dim3 grid((unsigned)((Vp + 127) / 128), 8), block(128);
  const double2* u = reinterpret_cast<const double2*>(U);
  switch (prec) {
    case P64: pack_links_kernel<P64><<<grid, block, 0, st>>>(u, out, nbr, lexp, lexq, Vp); break;
    case P32: pack_links_kernel<P32><<<grid, block, 0, st>>>(u, out, nbr, lexp, lexq, Vp); break;
    case P16: pack_links_kernel<P16><<<grid, block, 0, st>>>(u, out, nbr, lexp, lexq, Vp); break;
    default: pack_links_kernel<PB16><<<grid, block, 0, st>>>(u, out, nbr, lexp, lexq, Vp);
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_field_to(int prec, const void* src, void* dst, const int* map, long Vp,
                                 long nsrc, int Ls, cudaStream_t st) {
  dim3 grid((unsigned)((Vp + 127) / 128), Ls), block(128);
  const double2* s = reinterpret_cast<const double2*>(src);
  switch (prec) {
    case P64: pack_field_kernel<P64><<<grid, block, 0, st>>>(s, dst, map, Vp, nsrc, 1.0, 0); break;
    case P32: pack_field_kernel<P32><<<grid, block, 0, st>>>(s, dst, map, Vp, nsrc, 1.0, 0); break;
    case P16: pack_field_kernel<P16><<<grid, block, 0, st>>>(s, dst, map, Vp, nsrc, 1.0, 0); break;
    default: pack_field_kernel<PB16><<<grid, block, 0, st>>>(s, dst, map, Vp, nsrc, 1.0, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack_field_to(int prec, const void* src, void* dst, const int* map, long Vp,
                                   long ndst, int Ls, cudaStream_t st) {
  dim3 grid((unsigned)((Vp + 127) / 128), Ls), block(128);
  double2* d = reinterpret_cast<double2*>(dst);
  switch (prec) {
    case P64: unpack_field_kernel<P64><<<grid, block, 0, st>>>(src, d, map, Vp, ndst, 1.0, 0); break;
    case P32: unpack_field_kernel<P32><<<grid, block, 0, st>>>(src, d, map, Vp, ndst, 1.0, 0); break;
    case P16: unpack_field_kernel<P16><<<grid, block, 0, st>>>(src, d, map, Vp, ndst, 1.0, 0); break;
    default: unpack_field_kernel<PB16><<<grid, block, 0, st>>>(src, d, map, Vp, ndst, 1.0, 0);
  }
  return cudaGetLastError();
}

// The three post matrices of the stage kernels ([2][Ls][Ls] each, double): D+ M5op^-1
// (times b when c = 0), M5op^-dag D+^dag and D+^dag, plus M5op = alpha + beta K.
bool fifth_dim_matrices(int Ls, double M5, double mf, double b, double c,
                        std::vector<double>& dpm5i, std::vector<double>& m5idpt,
                        std::vector<double>& dpt, double* alpha, double* beta) {
  const double a = (4.0 - M5) * b + 1.0, be = (4.0 - M5) * c - 1.0;
  *alpha = a;
  *beta = be;
  dpm5i.clear();
  m5idpt.clear();
  dpt.clear();
  for (int chi = 0; chi < 2; chi++) {
    std::vector<double> K = kmat(Ls, mf, chi), D(Ls * Ls), M5m(Ls * Ls), M5i;
    for (int i = 0; i < Ls * Ls; i++) {
      const double id = (i % (Ls + 1) == 0) ? 1.0 : 0.0;
      D[i] = b * id + c * K[i];
      M5m[i] = a * id + be * K[i];
    }
    if (!invert(M5m, Ls, M5i)) return false;
    std::vector<double> DM = matmul(D, M5i, Ls);
    if (c == 0.0)
      for (auto& v : DM) v *= b;
    std::vector<double> MDt = matmul(transpose(M5i, Ls), transpose(D, Ls), Ls);
    std::vector<double> Dt = transpose(D, Ls);
    dpm5i.insert(dpm5i.end(), DM.begin(), DM.end());
    m5idpt.insert(m5idpt.end(), MDt.begin(), MDt.end());
    dpt.insert(dpt.end(), Dt.begin(), Dt.end());
  }
  return true;
}

}  // namespace dwf
