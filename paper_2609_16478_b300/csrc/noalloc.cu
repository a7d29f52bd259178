// Plan-free Dirichlet HOC Poisson solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns all device memory through its own pool, latency-critical
// loops where an allocation would synchronise the device, or environments
// that forbid allocation after start-up.  For them ahoc_poisson_noalloc
// runs the same solve as ahoc_poisson (DST-I along x [and y], the tridiagonal
// solve along the last axis, inverse DSTs) with its scratch -- the padded
// field, the twiddle and per-mode tables and the chunked-solve carries -- in
// one file-scope device array of kNoAllocBytes, which every GPU that loads
// the library keeps until the process exits.  Tables are rebuilt on the
// device at every call, so consecutive calls with different grids are fine;
// calls that overlap on the GPU (other streams, other threads) share the
// array and race.  Under lazy module loading (CUDA's default) the array is
// created on a device by the first call there, not when the library loads;
// its address is looked up once per device and must not be used across a
// cudaDeviceReset.
#include <cmath>
#include <mutex>
#include <string>

#include "ahoc.h"
#include "common.cuh"
#include "host.cuh"
#include "kernels.cuh"

namespace ahoc {
namespace {

constexpr size_t kNoAllocBytes = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {nullptr};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// tw[t] = exp(-2 pi i t / N) (t < N), sn[j] = sin(pi j / N) / 2 (j <= N/2)
__global__ void k_na_dst_tables(double* tw, double* sn, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N) {
    double s, c;
    sincospi(-2.0 * t / N, &s, &c);
    tw[2 * t] = c;
    tw[2 * t + 1] = s;
  }
  if (t <= N / 2) sn[t] = 0.5 * sinpi((double)t / N);
}

// (c, t) with exp(i pi x) = c (1 + i t), or = i c (1 + i t) when swap
__device__ void na_factor(double x, bool swap, double* out) {
  double sn, c;
  sincospi(x, &sn, &c);
  out[0] = swap ? sn : c;
  out[1] = swap ? -c / sn : sn / c;
}

// the entries after the first N of a DST table (layout at dst_tw_len)
__global__ void k_na_dst_stages(double* tw, int N) {
  const int M = N >> 1;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  int64_t off = N;
  for (int j = threadIdx.x; j <= N / 2; j += blockDim.x) {
    const double h = 0.5 * sinpi((double)j / N);
    tw[2 * (off + j)] = h + 0.25;
    tw[2 * (off + j) + 1] = h - 0.25;
  }
  off += N / 2 + 1;
  for (int Ns = (logM & 1) ? 2 : 1; Ns < M; Ns <<= 2) {
    if (Ns == 1) continue;
    for (int kk = threadIdx.x; kk < Ns; kk += blockDim.x) {
      const double x = -(double)kk / (2.0 * Ns);
      na_factor(x, dst_swap_w1(kk, Ns), tw + 2 * (off + kk));
      na_factor(2 * x, dst_swap_w2(kk, Ns), tw + 2 * (off + Ns + kk));
    }
    off += 2 * (int64_t)Ns;
  }
  for (int k = threadIdx.x; k <= M / 2; k += blockDim.x)
    na_factor(-2.0 * k / N, dst_swap_post(k, N), tw + 2 * (off + k));
  off += M / 2 + 1;
  for (int Ns = dst_r8_first_ns(logM); Ns < M; Ns <<= 3) {  // radix-8 stages
    for (int kk = threadIdx.x; kk < Ns; kk += blockDim.x) {
      const double x = -(double)kk / (4.0 * Ns);
      na_factor(x, false, tw + 2 * (off + kk));
      na_factor(2 * x, dst_swap_w1(kk, Ns), tw + 2 * (off + Ns + kk));
      na_factor(4 * x, dst_swap_w2(kk, Ns), tw + 2 * (off + 2 * Ns + kk));
      na_factor(x - 0.25, kk > 0, tw + 2 * (off + 3 * Ns + kk));
    }
    off += 4 * (int64_t)Ns;
  }
}

// sum of a few doubles with Neumaier compensation (the stencil-weight residue)
__device__ double na_fsum(const double* t, int n) {
  double s = 0.0, c = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = t[i], u = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - u) + x : (x - u) + s;
    s = u;
  }
  return s + c;
}

__device__ double na_ipow(double r, int n) {
  double out = 1.0, b = r;
  while (n > 0) {
    if (n & 1) out *= b;
    b *= b;
    n >>= 1;
  }
  return out;
}

// per-mode factors of the last-axis tridiagonal solve (the same quantities
// the plan computes on the host)
__global__ void k_na_modes(Geom g, Coefs cf, Mode<double>* modes) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (int64_t)nx * (g.dim == 3 ? (g.N[1] - 1) : 1);
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ncols) return;
  const int kx = 1 + (int)(m % nx);
  const int ky = (g.dim == 3) ? 1 + (int)(m / nx) : 0;
  const double cx = cospi((double)kx / g.N[0]);
  const double cy = (g.dim == 3) ? cospi((double)ky / g.N[1]) : 0.0;
  // u = 1 - cos(theta) = 2 sin^2(theta/2), without cancellation
  const double sx = sinpi((double)kx / (2.0 * g.N[0]));
  const double ux = 2.0 * sx * sx;
  const double sy = (g.dim == 3) ? sinpi((double)ky / (2.0 * g.N[1])) : 0.0;
  const double uy = 2.0 * sy * sy;
  auto L = [&](int dx, int dy, int dz) { return cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; };
  // a, b: diagonal and off-diagonal of the tridiagonal factor.  a + 2b is
  // written as S0 - 2 u (...) with S0 the (compensated) sum of the stencil
  // weights (zero in exact arithmetic, a rounding residue here) and
  // u = 1 - cos, so that 1 - 4 (b/a)^2 = (a + 2b)(a - 2b)/a^2 keeps its
  // relative accuracy for the lowest modes, as the plan's long-double
  // computation does
  double a, b, apb;
  if (g.dim == 2) {
    a = L(0, 0, 0) + 2 * cx * L(1, 0, 0);
    b = L(0, 1, 0) + 2 * cx * L(1, 1, 0);
    const double t[4] = {L(0, 0, 0), 2 * L(0, 1, 0), 2 * L(1, 0, 0), 4 * L(1, 1, 0)};
    apb = na_fsum(t, 4) - 2.0 * ux * (L(1, 0, 0) + 2 * L(1, 1, 0));
  } else {
    a = L(0, 0, 0) + 2 * cx * L(1, 0, 0) + 2 * cy * L(0, 1, 0) + 4 * cx * cy * L(1, 1, 0);
    b = L(0, 0, 1) + 2 * cx * L(1, 0, 1) + 2 * cy * L(0, 1, 1);
    const double t[7] = {L(0, 0, 0), 2 * L(0, 0, 1), 2 * L(1, 0, 0), 4 * L(1, 0, 1),
                         2 * L(0, 1, 0), 4 * L(0, 1, 1), 4 * L(1, 1, 0)};
    apb = na_fsum(t, 7) - 2.0 * ux * (L(1, 0, 0) + 2 * L(1, 0, 1) + 2 * L(1, 1, 0)) -
          2.0 * uy * (L(0, 1, 0) + 2 * L(0, 1, 1) + 2 * L(1, 1, 0)) + 4.0 * L(1, 1, 0) * ux * uy;
  }
  const int Nt = (g.dim == 3) ? g.N[2] : g.N[1];
  const int nt = Nt - 1;
  double scale = 2.0 / g.N[0];
  if (g.dim == 3) scale *= 2.0 / g.N[1];
  const double gam = -b / a;
  // = 1 - 4 gam^2 >= 0 for the diagonally dominant factors the host admits;
  // clamped so that rounding near |b/a| = 1/2 cannot give a NaN root
  const double disc = fmax(apb * (a - 2.0 * b) / (a * a), 0.0);
  const double r = 2 * gam / (1 + sqrt(disc));
  const double sigma = a / (1 + r * r);
  Mode<double> md;
  md.r = r;
  md.s = scale / sigma;
  const double r2N = na_ipow(r, 2 * Nt);
  md.kap = -r * (1 - r * r) / (1 - r2N);
  md.kapC = -r / (1 - r2N);
  md.q1 = 1.0 - r;
  if (r == 0.0) {
    md.rinv = 0;
    md.rj0 = 0;
    md.j0 = 0;
  } else {
    // the plan's cutoff: the last row where |r|^j is above 1e-18, so that the
    // seed K r^j0 of the boundary correction stays a normal number for any
    // right-hand side the solve can scale linearly
    const double lim = -18.0 * log(10.0) / log(fabs(r));
    const int j0 = (lim >= nt) ? nt : (lim < 0 ? 0 : (int)lim);
    md.rinv = 1.0 / r;
    md.rj0 = na_ipow(r, j0);
    md.j0 = j0;
  }
  modes[m] = md;
}

}  // namespace
}  // namespace ahoc

using namespace ahoc;

extern "C" ahoc_status ahoc_poisson_noalloc(int dim, const int64_t* N, const double* lo, const double* hi,
                                            const double* rhs, double* w, void* stream) {
  if (!rhs || !w) return host_fail(AHOC_EINVAL, "NULL argument");
  // 8-byte loads from a misaligned address would fault the context
  if ((reinterpret_cast<uintptr_t>(rhs) | reinterpret_cast<uintptr_t>(w)) & 7)
    return host_fail(AHOC_EINVAL, "device arrays of doubles must be 8-byte aligned");
  Geom g;
  ahoc_status s = host_make_geom(dim, N, lo, hi, &g);
  if (s != AHOC_OK) return s;
  const Coefs cf = host_make_coefs(g);
  const int nx = g.N[0] - 1;
  const int ny = (g.dim == 3) ? g.N[1] - 1 : 1;
  // every transverse mode must give a diagonally dominant tridiagonal factor
  for (int ky = 1; ky <= ny; ++ky)
    for (int kx = 1; kx <= nx; ++kx) {
      const double pi = 3.14159265358979323846;
      const double cx = std::cos(pi * kx / g.N[0]), cy = (g.dim == 3) ? std::cos(pi * ky / g.N[1]) : 0.0;
      auto L = [&](int dx, int dy, int dz) { return cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; };
      double a, b;
      if (g.dim == 2) {
        a = L(0, 0, 0) + 2 * cx * L(1, 0, 0);
        b = L(0, 1, 0) + 2 * cx * L(1, 1, 0);
      } else {
        a = L(0, 0, 0) + 2 * cx * L(1, 0, 0) + 2 * cy * L(0, 1, 0) + 4 * cx * cy * L(1, 1, 0);
        b = L(0, 0, 1) + 2 * cx * L(1, 0, 1) + 2 * cy * L(0, 1, 1);
      }
      if (!(std::fabs(b / a) < 0.5))
        return host_fail(AHOC_EUNSUPPORTED, "tridiagonal factor not diagonally dominant (mesh aspect ratio)");
    }
  // scratch layout inside the static array
  const bool chunked = host_tri_chunked(g);
  const int L = host_tri_chunk_len(g);
  const int64_t ncols = (int64_t)nx * ny;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t p = off;
    off += al256(bytes);
    return p;
  };
  const size_t o_field = take((size_t)g.npad * sizeof(double));
  const size_t o_twx = take(2 * (size_t)dst_tw_len(g.N[0]) * sizeof(double));
  const size_t o_snx = take(((size_t)g.N[0] / 2 + 1) * sizeof(double));
  const size_t o_twy = take(2 * (size_t)dst_tw_len(g.N[1]) * sizeof(double));
  const size_t o_sny = take(((size_t)g.N[1] / 2 + 1) * sizeof(double));
  const size_t o_modes = take((size_t)ncols * sizeof(Mode<double>));
  const size_t o_tri = take(chunked ? tri_chunked_scratch(g, L) * sizeof(double) : 0);
  const size_t o_rpow = take(chunked ? tri_powers_size(g, L) * sizeof(double) : 0);
  if (off > kNoAllocBytes) {
    const std::string msg = "ahoc_poisson_noalloc: this grid needs " + std::to_string(off) +
                            " bytes of scratch; the static scratch holds " + std::to_string(kNoAllocBytes) +
                            " bytes (16 MiB)";
    return host_fail(AHOC_EUNSUPPORTED, msg.c_str());
  }
  // the device address of the static array, looked up once per device with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return host_fail(AHOC_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return host_fail(AHOC_EUNSUPPORTED, "device ordinal beyond 63");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return host_fail(AHOC_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
      g_dev_ptr[dev] = ptr;
    }
    base = reinterpret_cast<unsigned char*>(g_dev_ptr[dev]);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* field = reinterpret_cast<double*>(base + o_field);
  double* twx = reinterpret_cast<double*>(base + o_twx);
  double* snx = reinterpret_cast<double*>(base + o_snx);
  double* twy = reinterpret_cast<double*>(base + o_twy);
  double* sny = reinterpret_cast<double*>(base + o_sny);
  Mode<double>* modes = reinterpret_cast<Mode<double>*>(base + o_modes);
  double* tri = reinterpret_cast<double*>(base + o_tri);
  double* rpow = reinterpret_cast<double*>(base + o_rpow);
#define NA_CK(call)                                                                              \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return host_fail(AHOC_ECUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)
  // the pad slots of the field must start at zero; the array keeps the last call's contents
  NA_CK(cudaMemsetAsync(field, 0, (size_t)g.npad * sizeof(double), st));
  k_na_dst_tables<<<(g.N[0] + 255) / 256, 256, 0, st>>>(twx, snx, g.N[0]);
  k_na_dst_stages<<<1, 256, 0, st>>>(twx, g.N[0]);
  NA_CK(cudaGetLastError());
  if (g.dim == 3) {
    k_na_dst_tables<<<(g.N[1] + 255) / 256, 256, 0, st>>>(twy, sny, g.N[1]);
    k_na_dst_stages<<<1, 256, 0, st>>>(twy, g.N[1]);
    NA_CK(cudaGetLastError());
  }
  k_na_modes<<<(unsigned)((ncols + 127) / 128), 128, 0, st>>>(g, cf, modes);
  NA_CK(cudaGetLastError());
  if (chunked) NA_CK(launch_tri_powers(g, modes, rpow, L, st));
  NA_CK(launch_unpack(g, field, rhs, st));
  NA_CK(launch_dst_x<double>(g, field, twx, snx, 1.0, st));
  if (g.dim == 3) NA_CK(launch_dst_y<double>(g, field, twy, sny, 1.0, st));
  if (chunked) NA_CK(launch_tri_chunked<double>(g, field, modes, modes, rpow, tri, L, st));
  else NA_CK(launch_tri<double>(g, field, modes, st));
  if (g.dim == 3) NA_CK(launch_dst_y<double>(g, field, twy, sny, 1.0, st));
  NA_CK(launch_dst_x<double>(g, field, twx, snx, 1.0, st));
  NA_CK(launch_pack(g, w, field, st));
#undef NA_CK
  return AHOC_OK;
}
