// C ABI entry points: handle lifecycle, dwf_apply, error reporting, shared helpers.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "engine.h"

namespace dwf {

static thread_local std::string g_last_error = "no error";

dwf_status set_error(dwf_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

dwf_status cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? DWF_ERR_NOMEM : DWF_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

dwf_status ensure_reduction(dwf_ctx* h, size_t partials, size_t counters) {
  if (h->red_partial_len < partials) {
    cudaFree(h->red_partial);
    h->red_partial = nullptr;
    DWF_CUDA(cudaMalloc(&h->red_partial, partials * sizeof(double)));
    h->red_partial_len = partials;
  }
  if (h->red_counter_len < counters) {
    cudaFree(h->red_counter);
    h->red_counter = nullptr;
    DWF_CUDA(cudaMalloc(&h->red_counter, counters * sizeof(unsigned)));
    DWF_CUDA(cudaMemset(h->red_counter, 0, counters * sizeof(unsigned)));
    h->red_counter_len = counters;
  }
  return DWF_OK;
}

RedArgs make_red(dwf_ctx* h, int cps, int op, double* res) {
  RedArgs r{};
  r.partial = h->red_partial;
  r.counter = h->red_counter;
  r.cps = cps;
  r.op = op;
  r.res = res;
  return r;
}

// Device view of a caller buffer: device pointers pass through; host buffers are copied into
// a named workspace buffer (when copy_in) and returned.
dwf_status stage_buffer(dwf_ctx* h, const char* name, const void* user, size_t bytes,
                        bool copy_in, void** dev) {
  if (is_device_ptr(user)) {
    *dev = const_cast<void*>(user);
    return DWF_OK;
  }
  DWF_TRY(h->ws->get(name, bytes, dev));
  if (copy_in) DWF_CUDA(cudaMemcpyAsync(*dev, user, bytes, cudaMemcpyHostToDevice, h->stream));
  return DWF_OK;
}

dwf_status finish_output(dwf_ctx* h, void* user, const void* dev, size_t bytes) {
  if (dev != user)
    DWF_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, h->stream));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

dwf_status check_device_error(dwf_ctx* h) {
  int e = 0;
  DWF_CUDA(cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  if (e) {
    // a CTA that gave up left its reduction segment unfinished: clear the counters so the
    // handle's next reductions start from zero
    DWF_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
    if (h->red_counter)
      DWF_CUDA(cudaMemsetAsync(h->red_counter, 0, h->red_counter_len * sizeof(unsigned),
                               h->stream));
    DWF_CUDA(cudaStreamSynchronize(h->stream));
    return set_error(DWF_ERR_TIMEOUT,
                     "a bounded device-side wait (TMA link staging or tensor-core completion) "
                     "gave up");
  }
  return DWF_OK;
}

static bool ls_supported(int Ls) {
  return Ls == 4 || Ls == 6 || Ls == 8 || Ls == 10 || Ls == 12 || Ls == 16;
}

}  // namespace dwf

using namespace dwf;

extern "C" {

const char* dwf_last_error(void) { return g_last_error.c_str(); }

const char* dwf_version(void) { return "dwf-gb300 0.2 (sm_103a)"; }

dwf_status dwf_set_option(dwf_t h, dwf_option opt, double value) {
  if (!h) return set_error(DWF_ERR_ARG, "null handle");
  switch (opt) {
    case DWF_OPT_WAIT_LIMIT_US:
      if (!(value >= 1.0 && value <= 1e7))
        return set_error(DWF_ERR_ARG, "wait limit must be in [1, 1e7] microseconds");
      h->wait_ns = (unsigned long long)(value * 1000.0);
      return DWF_OK;
    case DWF_OPT_TEST_WAIT_PROBE:
      h->wait_probe = value != 0.0 ? 1 : 0;
      return DWF_OK;
    default:
      return set_error(DWF_ERR_ARG, "unknown option");
  }
}

dwf_status dwf_create(dwf_t* handle, const int dims[4], int Ls, double M5, double mf, double b,
                      double c, const void* links, void* stream) {
  if (!handle || !dims || !links) return set_error(DWF_ERR_ARG, "null argument");
  *handle = nullptr;
  for (int m = 0; m < 4; m++)
    if (dims[m] < 2 || dims[m] % 2 != 0)
      return set_error(DWF_ERR_ARG, "lattice dims must be even and >= 2");
  if (!ls_supported(Ls)) return set_error(DWF_ERR_ARG, "Ls must be one of 4, 6, 8, 10, 12, 16");
  int dev = 0;
  DWF_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  DWF_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return set_error(DWF_ERR_ARG, "libdwf is built for sm_103a (GB300); device is sm_" +
                                      std::to_string(prop.major) + std::to_string(prop.minor));
  auto* h = new dwf_ctx();
  for (int m = 0; m < 4; m++) h->dims[m] = dims[m];
  h->Ls = Ls;
  h->M5 = M5;
  h->mf = mf;
  h->b = b;
  h->c = c;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->device = dev;
  // DWF_WAIT_LIMIT_US: initial limit of the handle's bounded device waits (profiler replays
  // slow kernels down; the default is 10 ms)
  if (const char* wl = getenv("DWF_WAIT_LIMIT_US")) {
    const double us = atof(wl);
    if (us >= 1.0 && us <= 1e7) h->wait_ns = (unsigned long long)(us * 1000.0);
  }
  h->ws = std::make_unique<Workspace>();
  const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  const size_t lbytes = (size_t)V * 4 * 9 * 16;
  dwf_status st = DWF_OK;
  if (cudaMalloc(&h->links_c128, lbytes) != cudaSuccess) {
    cudaGetLastError();
    dwf_destroy(h);
    return set_error(DWF_ERR_NOMEM, "links allocation failed");
  }
  if (cudaMalloc(&h->dev_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->dev_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    dwf_destroy(h);
    return set_error(DWF_ERR_NOMEM, "error flag allocation failed");
  }
  if (cudaMallocHost(&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    dwf_destroy(h);
    return set_error(DWF_ERR_NOMEM, "pinned allocation failed");
  }
  st = dwf_update_links(h, links);
  if (st == DWF_OK) st = build_matrices(h);
  Layout* lay = nullptr;
  if (st == DWF_OK) st = get_layout(h, dims, &lay);
  if (st == DWF_OK) st = ensure_reduction(h, lay->g.Vp / 32 * 2 + 64, lay->g.nblocks + 64);
  if (st != DWF_OK) {
    std::string msg = dwf_last_error();
    dwf_destroy(h);
    return set_error(st, msg);
  }
  *handle = h;
  return DWF_OK;
}

dwf_status dwf_update_links(dwf_t h, const void* links) {
  if (!h || !links) return set_error(DWF_ERR_ARG, "null argument");
  const long V = (long)h->dims[0] * h->dims[1] * h->dims[2] * h->dims[3];
  const size_t lbytes = (size_t)V * 4 * 9 * 16;
  DWF_CUDA(cudaMemcpyAsync(h->links_c128, links, lbytes, cudaMemcpyDefault, h->stream));
  for (auto& l : h->layouts)
    for (int p = 0; p < 4; p++) l->links_valid[p] = false;
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  return DWF_OK;
}

dwf_status dwf_apply(dwf_t h, dwf_op op, const void* in, void* out, dwf_prec prec) {
  if (!h || !in || !out) return set_error(DWF_ERR_ARG, "null argument");
  if (in == out) return set_error(DWF_ERR_ARG, "in and out must not alias");
  if ((int)prec < 0 || (int)prec > 3) return set_error(DWF_ERR_ARG, "bad precision");
  Layout* lay;
  DWF_TRY(get_layout(h, h->dims, &lay));
  OpEngine E;
  DWF_TRY(E.init(h, lay, (int)prec, false));
  const Geom& g = lay->g;
  const size_t fb = field_bytes(g, prec);
  const bool full = (op == DWF_OP_M || op == DWF_OP_MDAG);
  const size_t ubytes = (size_t)h->Ls * (full ? g.V : g.V / 2) * 12 * 16;
  void *din, *dout;
  DWF_TRY(stage_buffer(h, "apply_in", in, ubytes, true, &din));
  DWF_TRY(stage_buffer(h, "apply_out", out, ubytes, false, &dout));
  void *a, *b, *c, *d, *e, *f;
  DWF_TRY(h->ws->get("apply_a", fb, &a));
  DWF_TRY(h->ws->get("apply_b", fb, &b));
  DWF_TRY(h->ws->get("apply_c", fb, &c));
  DWF_TRY(h->ws->get("apply_d", fb, &d));
  DWF_TRY(h->ws->get("apply_e", fb, &e));
  DWF_TRY(h->ws->get("apply_f", fb, &f));
  RedArgs none{};
  switch (op) {
    case DWF_OP_M:
    case DWF_OP_MDAG:
      DWF_TRY(pack_full(h, lay, din, a, b, prec));
      DWF_TRY(E.full(a, b, c, d, e, f, op == DWF_OP_MDAG));
      DWF_TRY(unpack_full(h, lay, e, f, prec, dout));
      break;
    case DWF_OP_MPC:
      DWF_TRY(pack_even(h, lay, din, a, prec, 1.0));
      DWF_TRY(E.mpc(a, b, c, d, EPI_STORE, none, nullptr));
      DWF_TRY(unpack_even(h, lay, d, prec, dout, 1.0));
      break;
    case DWF_OP_MPC_DAG:
      DWF_TRY(pack_even(h, lay, din, a, prec, 1.0));
      DWF_TRY(E.mpcdag(a, c, d, EPI_STORE, nullptr, nullptr, none, nullptr));
      DWF_TRY(unpack_even(h, lay, d, prec, dout, 1.0));
      break;
    case DWF_OP_MDAGM:
      DWF_TRY(pack_even(h, lay, din, a, prec, 1.0));
      DWF_TRY(E.mpc(a, b, c, d, EPI_STORE, none, nullptr));
      DWF_TRY(E.mpcdag(d, c, e, EPI_STORE, nullptr, nullptr, none, nullptr));
      DWF_TRY(unpack_even(h, lay, e, prec, dout, 1.0));
      break;
    default:
      return set_error(DWF_ERR_ARG, "unknown operator");
  }
  return finish_output(h, out, dout, ubytes);
}

dwf_status dwf_profile_enable(dwf_t h, int on) {
  if (!h) return set_error(DWF_ERR_ARG, "null handle");
  h->prof.on = on != 0;
  return DWF_OK;
}

dwf_status dwf_profile_read(dwf_t h, dwf_kernel_profile* out, int capacity, int* n) {
  if (!h || !n) return set_error(DWF_ERR_ARG, "null argument");
  DWF_CUDA(cudaStreamSynchronize(h->stream));
  Profiler& P = h->prof;
  std::vector<dwf_kernel_profile> acc(P.names.size());
  for (size_t i = 0; i < P.names.size(); i++) {
    memset(&acc[i], 0, sizeof(dwf_kernel_profile));
    snprintf(acc[i].name, sizeof(acc[i].name), "%s", P.names[i].c_str());
  }
  for (const auto& r : P.recs) {
    float ms = 0.f;
    DWF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    dwf_kernel_profile& k = acc[r.cls];
    k.launches++;
    k.ms_total += ms;
    k.bytes_total += r.bytes;
    k.flops_total += r.flops;
  }
  int m = 0;
  for (auto& k : acc)
    if (k.launches && m < capacity && out) out[m++] = k;
  *n = m;
  P.recs.clear();
  P.used = 0;
  return DWF_OK;
}

void dwf_destroy(dwf_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  h->layouts.clear();
  h->ws.reset();
  for (int i = 0; i < 2; i++) {
    cudaFree(h->mats.d_dp[i]);
    cudaFree(h->mats.d_dpt[i]);
    cudaFree(h->mats.d_dpm5i[i]);
    cudaFree(h->mats.d_m5idpt[i]);
  }
  for (int i = 0; i < 3; i++) cudaFree(h->mats.d_post_h[i]);
  cudaFree(h->dev_err);
  cudaFree(h->links_c128);
  cudaFree(h->red_partial);
  cudaFree(h->red_counter);
  cudaFree(h->scal);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  delete h;
}

}  // extern "C"
