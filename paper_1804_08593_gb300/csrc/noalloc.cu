// A = Mpc^dag Mpc without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the operator: a
// host runtime that owns every device buffer up front (a fixed memory budget or a pool that
// must not grow during a run), a caller that is itself running inside a region where
// cudaMalloc/cudaFree would synchronise the device or break its own bookkeeping, or an
// embedding that only hands the library raw device pointers.  dwf_mdagm_noalloc serves them:
// it takes its inputs and output from the caller and keeps everything else (neighbour tables,
// packed links, the fifth-dimension matrices, the packed input and the intermediate fields)
// in one file-scope __device__ array of fixed size, DWF_NOALLOC_SCRATCH_BYTES.  Every GPU that
// loads the library holds that array until the process exits.
//
// The host cannot use the array's symbol as a device address, so the first call on a device
// (with that device current) looks the address up once with cudaGetSymbolAddress and caches
// it; make that first call before any stream capture.  All calls share the array and leave
// their data in it; calls whose executions overlap on the GPU (different streams, or the same
// stream from several host threads) race on it and must be serialised by the caller.  The
// fifth-dimension matrices reach the device as a kernel argument (no host buffer outlives the
// call), and a bounded device wait that gives up turns the whole output into NaN.
#include <mutex>
#include <vector>

#include "engine.h"

namespace dwf {

cudaError_t launch_pack_links_to(int prec, const void* U, void* out, const uint32_t* nbr,
                                 const int* lexp, const int* lexq, long Vp, cudaStream_t st);
cudaError_t launch_pack_field_to(int prec, const void* src, void* dst, const int* map, long Vp,
                                 long nsrc, int Ls, cudaStream_t st);
cudaError_t launch_unpack_field_to(int prec, const void* src, void* dst, const int* map, long Vp,
                                   long ndst, int Ls, cudaStream_t st);
bool fifth_dim_matrices(int Ls, double M5, double mf, double b, double c,
                        std::vector<double>& dpm5i, std::vector<double>& m5idpt,
                        std::vector<double>& dpt, double* alpha, double* beta);

namespace {

constexpr size_t kScratchBytes = DWF_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
dwf_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(DWF_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_scratch)");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return DWF_OK;
}

// Neighbour and site tables of the plain checkerboard order (one block = the lattice).
__global__ void plain_tables_kernel(int X, int Y, int Z, int T, long Vh, long Vp, uint32_t* nbr0,
                                    uint32_t* nbr1, int* lex0, int* lex1, int* cbe) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (j >= Vp) return;
  uint32_t* nbr = p ? nbr1 : nbr0;
  int* lex = p ? lex1 : lex0;
  if (j >= Vh) {
    for (int d = 0; d < 8; d++) nbr[d * Vp + j] = 0u;
    lex[j] = -1;
    if (p == 0) cbe[j] = -1;
    return;
  }
  const int hx = X / 2;
  long r = j;
  const int jx = (int)(r % hx);
  r /= hx;
  const int y = (int)(r % Y);
  r /= Y;
  const int z = (int)(r % Z);
  const int t = (int)(r / Z);
  const int x = 2 * jx + ((p + y + z + t) & 1);
  const int L[4] = {X, Y, Z, T};
  const long lx = x + (long)X * (y + (long)Y * (z + (long)Z * t));
  lex[j] = (int)lx;
  if (p == 0) cbe[j] = (int)(lx / 2);
  for (int d = 0; d < 8; d++) {
    int c[4] = {x, y, z, t};
    const int mu = d >> 1;
    c[mu] = (c[mu] + ((d & 1) ? L[mu] - 1 : 1)) % L[mu];
    nbr[d * Vp + j] =
        (uint32_t)(c[0] / 2 + (long)hx * (c[1] + (long)Y * (c[2] + (long)Z * c[3])));
  }
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// The three per-chirality fifth-dimension matrices ([3][2][Ls][Ls], Ls <= 16) travel to the
// device inside the kernel's parameter block, so no host buffer is read after the call
// returns and no host-to-device copy is queued.
struct MatParam {
  double v[3 * 2 * 16 * 16];
};
static_assert(sizeof(MatParam) <= 32000, "kernel parameter block limit");

__global__ void write_mats_kernel(const MatParam m, int n, int as_double, void* dst) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (as_double) static_cast<double*>(dst)[i] = m.v[i];
    else static_cast<float*>(dst)[i] = (float)m.v[i];
  }
}

// A bounded device wait that gave up (TMA link staging, tensor-core completion) sets *status;
// then every element of the output becomes a quiet NaN, so that a timed-out call cannot pass
// for a valid result (the call itself returns before the kernels run).
__global__ void poison_if_error_kernel(const int* status, double* out, long n) {
  if (*status == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    out[i] = nan;
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_mdagm_noalloc(const int dims[4], int Ls, double M5, double mf,
                                        double b, double c, const void* links, const void* in,
                                        void* out, dwf_prec prec, void* stream) {
  if (!dims || !links || !in || !out) return set_error(DWF_ERR_ARG, "null argument");
  if (in == out) return set_error(DWF_ERR_ARG, "in and out must not alias");
  if ((int)prec < 0 || (int)prec > 3) return set_error(DWF_ERR_ARG, "bad precision");
  if (!(Ls == 4 || Ls == 6 || Ls == 8 || Ls == 10 || Ls == 12 || Ls == 16))
    return set_error(DWF_ERR_ARG, "Ls must be one of 4, 6, 8, 10, 12, 16");
  for (int m = 0; m < 4; m++)
    if (dims[m] < 2 || dims[m] % 2 != 0)
      return set_error(DWF_ERR_ARG, "lattice dims must be even and >= 2");
  if (!is_device_ptr(links) || !is_device_ptr(in) || !is_device_ptr(out))
    return set_error(DWF_ERR_ARG, "dwf_mdagm_noalloc takes device pointers only");
  int dev = 0;
  DWF_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  DWF_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return set_error(DWF_ERR_ARG, "libdwf is built for sm_103a (GB300)");

  const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  const long Vh = V / 2;
  const long Vp = (Vh + 31) / 32 * 32;
  const int P = (int)prec;
  const size_t acc = (P == P64) ? sizeof(double) : sizeof(float);
  const size_t link_chunks = P == P64 ? 9 : P == P32 ? 5 : 3;   // 16-byte chunks per link
  const size_t fb = (size_t)Ls * Vp * 24 * real_bytes(P);
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += align256(n);
    return o;
  };
  const size_t o_nbr0 = take(8 * Vp * 4), o_nbr1 = take(8 * Vp * 4);
  const size_t o_lex0 = take(Vp * 4), o_lex1 = take(Vp * 4), o_cbe = take(Vp * 4);
  const size_t o_l0 = take(8 * link_chunks * 16 * Vp), o_l1 = take(8 * link_chunks * 16 * Vp);
  const size_t o_m = take(3 * 2 * Ls * Ls * acc);
  const size_t o_status = take(sizeof(int));
  size_t o_f[6];
  for (int i = 0; i < 6; i++) o_f[i] = take(fb);
  if (off > kScratchBytes)
    return set_error(DWF_ERR_ARG, "lattice too large for dwf_mdagm_noalloc: needs " +
                                      std::to_string(off) + " bytes of scratch, the maximum is " +
                                      std::to_string(kScratchBytes));
  unsigned char* S;
  DWF_TRY(scratch_address(dev, &S));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  std::vector<double> dpm5i, m5idpt, dpt;
  double ma, mb;
  if (!fifth_dim_matrices(Ls, M5, mf, b, c, dpm5i, m5idpt, dpt, &ma, &mb))
    return set_error(DWF_ERR_ARG, "M5op is singular");
  MatParam mp;
  for (int w = 0; w < 3; w++) {
    const std::vector<double>& m = w == 0 ? dpm5i : w == 1 ? m5idpt : dpt;
    for (int i = 0; i < 2 * Ls * Ls; i++) mp.v[w * 2 * Ls * Ls + i] = m[i];
  }
  write_mats_kernel<<<1, 256, 0, st>>>(mp, 3 * 2 * Ls * Ls, acc == sizeof(double) ? 1 : 0,
                                       S + o_m);
  DWF_CUDA(cudaGetLastError());
  int* status = reinterpret_cast<int*>(S + o_status);
  DWF_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));

  uint32_t* nbr[2] = {reinterpret_cast<uint32_t*>(S + o_nbr0), reinterpret_cast<uint32_t*>(S + o_nbr1)};
  int* lex[2] = {reinterpret_cast<int*>(S + o_lex0), reinterpret_cast<int*>(S + o_lex1)};
  int* cbe = reinterpret_cast<int*>(S + o_cbe);
  void* lk[2] = {S + o_l0, S + o_l1};
  void* f[6];
  for (int i = 0; i < 6; i++) f[i] = S + o_f[i];
  {
    dim3 grid((unsigned)((Vp + 127) / 128), 2), block(128);
    plain_tables_kernel<<<grid, block, 0, st>>>(dims[0], dims[1], dims[2], dims[3], Vh, Vp,
                                                nbr[0], nbr[1], lex[0], lex[1], cbe);
    DWF_CUDA(cudaGetLastError());
  }
  for (int p = 0; p < 2; p++)
    DWF_CUDA(launch_pack_links_to(P, links, lk[p], nbr[p], lex[p], lex[1 - p], Vp, st));
  DWF_CUDA(launch_pack_field_to(P, in, f[0], cbe, Vp, Vh, Ls, st));

  const bool trivial = (c == 0.0);
  const unsigned char* M = S + o_m;
  const void* post_a = M;
  const void* post_ad = M + 2 * Ls * Ls * acc;
  const void* post_bd = M + 2 * 2 * Ls * Ls * acc;
  auto base = [&](int par) {
    StageArgs a{};
    a.links = lk[par];
    a.nbr = nbr[par];
    a.Vp = a.Vp_in = a.Vp_halo = a.Vp_link = Vp;
    a.Vhb = (int)Vh;
    a.Vhb_pad = (int)Vp;
    a.seg_cps = (int)(Vp / 32);
    a.hop_scale = 1.0;
    a.mf = mf;
    a.l_alpha = ma;
    a.l_beta = mb;
    a.epi = EPI_STORE;
    a.err = status;
    return a;
  };
  // fields: f0 = x, f1 = D+ x, f2 = t (odd), f3 = y = Mpc x, f4 = s (odd), f5 = A x
  const void* xin = f[0];
  if (!trivial) {
    VecArgs v{};
    v.p = f[0];
    v.u = f[1];
    v.Vp = Vp;
    v.Vhb = (int)Vh;
    v.Vhb_pad = (int)Vp;
    v.seg_cps = (int)(Vp / 32);
    v.do_u = 1;
    v.db = b;
    v.dc = c;
    v.mf = mf;
    DWF_CUDA(launch_vec(P, v, Ls, st));
    xin = f[1];
  }
  StageArgs s1 = base(1);
  s1.in = xin;
  s1.out = f[2];
  s1.post = post_a;
  DWF_CUDA(launch_stage_prec(P, s1, Ls, false, false, st));
  StageArgs s2 = base(0);
  s2.in = f[2];
  s2.out = f[3];
  s2.in2 = f[0];
  s2.local_mode = LOC_M5;
  s2.hop_scale = -0.25;
  DWF_CUDA(launch_stage_prec(P, s2, Ls, false, false, st));
  StageArgs s3 = base(1);
  s3.in = f[3];
  s3.out = f[4];
  s3.post = post_ad;
  DWF_CUDA(launch_stage_prec(P, s3, Ls, true, false, st));
  StageArgs s4 = base(0);
  s4.in = f[4];
  s4.out = f[5];
  s4.in2 = f[3];
  s4.local_mode = LOC_M5DAG;
  if (trivial) {
    s4.hop_scale = -0.25 * b;
  } else {
    s4.hop_scale = -0.25;
    s4.post = post_bd;
  }
  DWF_CUDA(launch_stage_prec(P, s4, Ls, true, false, st));
  DWF_CUDA(launch_unpack_field_to(P, f[5], out, cbe, Vp, Vh, Ls, st));
  poison_if_error_kernel<<<64, 256, 0, st>>>(status, static_cast<double*>(out),
                                             (long)Ls * Vh * 24);
  DWF_CUDA(cudaGetLastError());
  return DWF_OK;
}
