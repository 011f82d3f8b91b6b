// lgt_noalloc.cu -- exact F / theta / plaquette measurement that allocates
// nothing (see lgt_measure_noalloc in include/lgt.h).
//
// lgt_measure needs a context, and a context owns device buffers that
// lgt_create obtains with cudaMalloc.  Some callers cannot allocate: an
// application that owns every byte of device memory through its own memory
// plan or pool and may not have a library take memory behind its back, or code
// that measures a field from a place where no allocation may happen (between
// the steps of a fixed memory budget).  For them this variant reads the links
// directly in the public layout from the caller's device buffer, writes its
// results to the caller's device buffer, and keeps its reduction scratch in
// one file-scope __device__ array of a fixed size.
#include <cuda_runtime.h>

#include <mutex>

#include "lgt_api_internal.h"

namespace {

constexpr int kBlocksPerSlice = 16;  // fixed grid: 16 blocks per timeslice
constexpr int kThreads = 256;
constexpr int kMaxSlices = 1024;     // largest N_t the scratch array holds
constexpr int kNV = 5;               // quantities reduced per site (see below)
constexpr int kMaxDevices = 64;

// The shared scratch: per-block partial sums, per-slice sums and the counters
// of the last-block reductions.  About 700 KB, held by every device that loads
// the library until the process exits.
struct NoAllocScratch {
  double partial[kMaxSlices][kBlocksPerSlice][kNV];
  double slice_sum[kMaxSlices][kNV];
  unsigned counter[kMaxSlices];
  unsigned glob;
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

#define RE(a, b) (2 * (3 * (a) + (b)))
#define IM(a, b) (2 * (3 * (a) + (b)) + 1)

struct Dims {
  int nt, n3, n2, n1;
  long long vs;  // sites per timeslice
};

__device__ __forceinline__ long long lex_of(const Dims &d, int x1, int x2, int x3, int t) {
  return (long long)x1 + (long long)d.n1 * (x2 + (long long)d.n2 * (x3 + (long long)d.n3 * t));
}

__device__ __forceinline__ void load_aos(const double *links, long long lex, int mu, double u[18]) {
  const double *src = links + ((size_t)lex * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 18; k++) u[k] = src[k];
}

// X += s (U - U^dagger)
__device__ __forceinline__ void add_antiherm(double X[18], const double u[18], double s) {
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      X[RE(a, b)] += s * (u[RE(a, b)] - u[RE(b, a)]);
      X[IM(a, b)] += s * (u[IM(a, b)] + u[IM(b, a)]);
    }
}

// tr[D D^dagger], D the traceless part of X/(2i) (X anti-Hermitian)
__device__ __forceinline__ double delta_norm(const double X[18]) {
  const double d0 = 0.5 * X[IM(0, 0)], d1 = 0.5 * X[IM(1, 1)], d2 = 0.5 * X[IM(2, 2)];
  const double m = (d0 + d1 + d2) / 3.0;
  double s = (d0 - m) * (d0 - m) + (d1 - m) * (d1 - m) + (d2 - m) * (d2 - m);
  for (int a = 0; a < 3; a++)
    for (int b = a + 1; b < 3; b++) s += 0.5 * (X[RE(a, b)] * X[RE(a, b)] + X[IM(a, b)] * X[IM(a, b)]);
  return s;
}

__device__ __forceinline__ void matmul(const double a[18], const double b[18], double c[18]) {
  for (int r = 0; r < 3; r++)
    for (int s = 0; s < 3; s++) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < 3; k++) {
        re += a[RE(r, k)] * b[RE(k, s)] - a[IM(r, k)] * b[IM(k, s)];
        im += a[RE(r, k)] * b[IM(k, s)] + a[IM(r, k)] * b[RE(k, s)];
      }
      c[RE(r, s)] = re;
      c[IM(r, s)] = im;
    }
}

// Per site: [0] sum_mu Re tr U_mu, [1] the same over mu = 1..3, [2] tr Delta^2
// (4-D), [3] tr Delta_s^2 (spatial), [4] sum of the six plaquettes Re tr U_P.
__global__ void __launch_bounds__(kThreads) k_measure_noalloc(Dims d, const double *links, double *out) {
  NoAllocScratch &S = g_noalloc_scratch;
  const int t = blockIdx.y;
  double v[kNV] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long k = (long long)blockIdx.x * kThreads + threadIdx.x; k < d.vs; k += (long long)kBlocksPerSlice * kThreads) {
    const int x1 = (int)(k % d.n1);
    const long long r = k / d.n1;
    const int x2 = (int)(r % d.n2);
    const int x3 = (int)(r / d.n2);
    const int xc[4] = {t, x1, x2, x3};  // coordinate along each direction mu
    const int nn[4] = {d.nt, d.n1, d.n2, d.n3};
    const long long lex = lex_of(d, x1, x2, x3, t);
    double XL[18], XS[18];
    for (int e = 0; e < 18; e++) XL[e] = XS[e] = 0.0;
    long long fwd_nb[4];
    for (int mu = 0; mu < 4; mu++) {
      int y[4] = {xc[0], xc[1], xc[2], xc[3]};
      y[mu] = (y[mu] + nn[mu] - 1) % nn[mu];
      const long long back = lex_of(d, y[1], y[2], y[3], y[0]);
      y[mu] = (xc[mu] + 1) % nn[mu];
      fwd_nb[mu] = lex_of(d, y[1], y[2], y[3], y[0]);
      double u[18];
      load_aos(links, lex, mu, u);
      const double rt = u[RE(0, 0)] + u[RE(1, 1)] + u[RE(2, 2)];
      v[0] += rt;
      add_antiherm(XL, u, 1.0);
      if (mu > 0) {
        v[1] += rt;
        add_antiherm(XS, u, 1.0);
      }
      load_aos(links, back, mu, u);
      add_antiherm(XL, u, -1.0);
      if (mu > 0) add_antiherm(XS, u, -1.0);
    }
    v[2] += delta_norm(XL);
    v[3] += delta_norm(XS);
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        double a[18], b[18], c[18], e[18], m1[18], m2[18];
        load_aos(links, lex, mu, a);
        load_aos(links, fwd_nb[mu], nu, b);
        load_aos(links, fwd_nb[nu], mu, c);
        load_aos(links, lex, nu, e);
        matmul(a, b, m1);
        matmul(e, c, m2);
        double s = 0.0;
        for (int q = 0; q < 18; q++) s += m1[q] * m2[q];
        v[4] += s;
      }
  }
  // fixed-order block sum
  __shared__ double warp_part[kNV][kThreads / 32];
  __shared__ int am_last, am_final;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < kNV; q++) {
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    if (lane == 0) warp_part[q][warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < kNV; q++) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; w++) s += warp_part[q][w];
      S.partial[t][blockIdx.x][q] = s;
    }
    __threadfence();
    am_last = atomicAdd(&S.counter[t], 1u) == (unsigned)kBlocksPerSlice - 1;
  }
  __syncthreads();
  if (!am_last || threadIdx.x != 0) return;
  // last block of slice t: its slice sums, in block order
  __threadfence();
  for (int q = 0; q < kNV; q++) {
    double s = 0.0;
    for (int b = 0; b < kBlocksPerSlice; b++) s += __ldcg(&S.partial[t][b][q]);
    S.slice_sum[t][q] = s;
  }
  const double vs = (double)d.vs;
  out[8 + t] = S.slice_sum[t][1] / (9.0 * vs);
  out[8 + d.nt + t] = S.slice_sum[t][3] / (3.0 * vs);
  S.counter[t] = 0u;
  __threadfence();
  am_final = atomicAdd(&S.glob, 1u) == (unsigned)d.nt - 1;
  if (!am_final) return;
  // last slice: totals in slice order
  __threadfence();
  double s[kNV] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double fsum = 0.0, tmax = 0.0, tsum = 0.0;
  for (int tt = 0; tt < d.nt; tt++) {
    for (int q = 0; q < kNV; q++) s[q] += __ldcg(&S.slice_sum[tt][q]);
    const double ft = __ldcg(&S.slice_sum[tt][1]) / (9.0 * vs);
    const double th = __ldcg(&S.slice_sum[tt][3]) / (3.0 * vs);
    fsum += ft;
    tsum += th;
    tmax = th > tmax ? th : tmax;
  }
  const double vol = vs * d.nt;
  out[0] = s[0] / (12.0 * vol);  // F, Landau
  out[1] = s[2] / (3.0 * vol);   // theta, Landau
  out[2] = s[4] / (18.0 * vol);  // average plaquette
  out[3] = fsum / d.nt;          // mean F_t, Coulomb
  out[4] = tmax;                 // max theta_t, Coulomb
  out[5] = tsum / d.nt;          // mean theta_t, Coulomb
  out[6] = 0.0;
  out[7] = 0.0;
  S.glob = 0u;
}

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];  // device address of the scratch, per device

}  // namespace

extern "C" lgt_status lgt_measure_noalloc(const int32_t dims[4], const double *links_device, double *out_device,
                                          void *cuda_stream) {
  if (!dims || !links_device || !out_device) {
    lgt_set_error("lgt_measure_noalloc: NULL argument");
    return LGT_EINVAL;
  }
  for (int k = 0; k < 4; k++)
    if (dims[k] < 2 || (dims[k] & 1)) {
      lgt_set_error("lgt_measure_noalloc: dims[%d] = %d must be even and >= 2", k, dims[k]);
      return LGT_EINVAL;
    }
  if (dims[0] > kMaxSlices) {
    lgt_set_error("lgt_measure_noalloc: N_t = %d exceeds the maximum of %d timeslices its fixed scratch holds",
                  dims[0], kMaxSlices);
    return LGT_EINVAL;
  }
  const double vs = (double)dims[1] * dims[2] * dims[3];
  if (vs * dims[0] > 4.0e9) {
    lgt_set_error("lgt_measure_noalloc: lattice too large");
    return LGT_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    lgt_set_error("lgt_measure_noalloc: no usable current device (%s)", cudaGetErrorString(e));
    return LGT_ECUDA;
  }
  void *scratch = nullptr;
  {
    // first call on this device: look up the device address of the scratch
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        lgt_set_error("lgt_measure_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return LGT_ECUDA;
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the counters start from zero on every call (a previous call's state is not trusted)
  NoAllocScratch *S = (NoAllocScratch *)scratch;
  e = cudaMemsetAsync(&S->counter[0], 0, sizeof(unsigned) * (kMaxSlices + 1), st);
  if (e != cudaSuccess) {
    lgt_set_error("lgt_measure_noalloc: %s", cudaGetErrorString(e));
    return LGT_ECUDA;
  }
  Dims d = {dims[0], dims[1], dims[2], dims[3], (long long)dims[1] * dims[2] * dims[3]};
  k_measure_noalloc<<<dim3(kBlocksPerSlice, dims[0]), kThreads, 0, st>>>(d, links_device, out_device);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    lgt_set_error("lgt_measure_noalloc: launch failed: %s", cudaGetErrorString(e));
    return LGT_ECUDA;
  }
  return LGT_OK;
}
