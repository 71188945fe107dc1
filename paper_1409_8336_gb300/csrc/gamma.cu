// 3-D gamma index (Low et al.) between two dose grids, the dose-comparison metric
// the paper computes on the GPU (Sec. II.D).  Global dose criterion (a percentage
// of the reference maximum), distance-to-agreement criterion, evaluated on the
// grid without interpolation:
//
//   gamma^2(v) = min over voxels w with |r_w - r_v| <= search of
//                |r_w - r_v|^2 / dta^2 + (D_eval(w) - D_ref(v))^2 / tol^2
//
// for every reference voxel v whose dose exceeds threshold * max(D_ref).
//
// The offsets w - v inside the search sphere are listed once on the host, sorted
// by their distance term.  A voxel's scan stops at the first offset whose distance
// term alone reaches the minimum found so far: every later value is at least that
// large, so the minimum is the exhaustive one, bit for bit (rounding is monotone).
// Most voxels of a dose comparison stop after a few offsets.  An offset whose value
// is bounded below by the minimum so far skips the division (FP64 arithmetic is the
// scarce resource here).
#include <cmath>
#include <cstddef>
#include <cstdint>

#include "pmc_kernels.cuh"

namespace pmc {
namespace {

// Doubles compared as unsigned integers: negative values bit-inverted, non-negative
// ones with the sign bit set, so that integer order is numeric order.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Maximum of the reference dose: four voxels per thread and iteration (two 16-byte
// loads in flight), the ragged tail by the first threads.
__global__ void dose_max_kernel(const double* __restrict__ d, long long n, bool vec, GammaHead* head) {
  double m = -INFINITY;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long n4 = vec ? n / 4 : 0;
  const double2* d2 = reinterpret_cast<const double2*>(d);
  for (long long q = t; q < n4; q += stride) {
    const double2 a = __ldg(d2 + 2 * q), b = __ldg(d2 + 2 * q + 1);
    m = fmax(m, fmax(fmax(a.x, a.y), fmax(b.x, b.y)));
  }
  for (long long i = 4 * n4 + t; i < n; i += stride) m = fmax(m, d[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(&head->max_key, order_key(m));
}

struct GammaCtx {
  const double* ev;
  const GammaOffset* off;
  int n_off, nx, ny, nz;
  long long nxy;
  double tol2, inv_tol2;
};

// gamma^2 of reference voxel v (dose d): the sorted offsets, stopping at the first whose
// distance term alone reaches the minimum so far.
__device__ __forceinline__ double gamma2_at(const GammaCtx c, long long v, double d) {
  const int iz = static_cast<int>(v / c.nxy);
  const int rem = static_cast<int>(v - iz * c.nxy);
  const int iy = rem / c.nx, ix = rem - iy * c.nx;
  double g2 = INFINITY;
  for (int i = 0; i < c.n_off; ++i) {
    const GammaOffset o = c.off[i];
    if (o.r_term >= g2) break;
    const int jx = ix + o.kx, jy = iy + o.ky, jz = iz + o.kz;
    if (static_cast<unsigned>(jx) >= static_cast<unsigned>(c.nx) ||
        static_cast<unsigned>(jy) >= static_cast<unsigned>(c.ny) || static_cast<unsigned>(jz) >= static_cast<unsigned>(c.nz))
      continue;
    const double dd = __ldg(c.ev + jz * c.nxy + static_cast<long long>(jy) * c.nx + jx) - d;
    const double dd2 = __dmul_rn(dd, dd);
    // dd2 * (1/tol^2) is within 3 ulp of the quotient, so this lower bound of the value
    // rules the offset out without the (slow, FP64) correctly rounded division
    if (__dadd_rn(o.r_term, __dmul_rn(__dmul_rn(dd2, c.inv_tol2), 1.0 - 1e-14)) >= g2) continue;
    const double val = __dadd_rn(o.r_term, __ddiv_rn(dd2, c.tol2));
    g2 = val < g2 ? val : g2;
  }
  return g2;
}

// One pass over the reference grid, four voxels per thread when the pointers allow
// 16-byte access.  Blocks claim chunks of 256 quads from a counter: the voxels above
// the threshold cluster where the beams are, and a static split would leave most SMs
// idle while a few scan them.  Counts of evaluated and passing voxels are reduced per
// warp.  The scan's cost is FP64 instructions (a GB300 SM retires few per clock), which
// the sorted offsets, the early stop and the division skip keep down.
__global__ void __launch_bounds__(256) gamma_kernel(const double* __restrict__ ref, const double* __restrict__ ev,
                                                    int nx, int ny, int nz, bool vec, GammaHead* head,
                                                    const GammaOffset* __restrict__ off, double dose_pct,
                                                    double threshold, float* __restrict__ gamma) {
  const double dmax = key_value(head->max_key);
  const double tol = dose_pct / 100.0 * dmax;
  const double thr = threshold * dmax;
  GammaCtx c;
  c.ev = ev;
  c.off = off;
  c.n_off = head->n_off;
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.nxy = static_cast<long long>(nx) * ny;
  c.tol2 = tol * tol;
  c.inv_tol2 = 1.0 / c.tol2;
  const long long n = c.nxy * nz;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long n4 = vec ? n / 4 : 0;
  unsigned long long n_eval = 0, n_pass = 0;
  const double2* r2 = reinterpret_cast<const double2*>(ref);
  auto one = [c, thr, &n_eval, &n_pass](long long v, double d) {
    if (!(d > thr)) return -1.0f;
    const double g2 = gamma2_at(c, v, d);
    ++n_eval;
    n_pass += g2 <= 1.0 + 1e-12;
    return static_cast<float>(sqrt(g2));
  };
  __shared__ long long s_chunk;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_chunk = static_cast<long long>(atomicAdd(&head->work, 1ull));
    __syncthreads();
    const long long q0 = s_chunk * blockDim.x;
    if (q0 >= n4) break;
    const long long q = q0 + threadIdx.x;
    if (q < n4) {
      const double2 a = __ldg(r2 + 2 * q), b = __ldg(r2 + 2 * q + 1);
      const float4 g = make_float4(one(4 * q, a.x), one(4 * q + 1, a.y), one(4 * q + 2, b.x), one(4 * q + 3, b.y));
      if (gamma) reinterpret_cast<float4*>(gamma)[q] = g;
    }
  }
  for (long long v = 4 * n4 + t; v < n; v += stride) {
    const float g = one(v, ref[v]);
    if (gamma) gamma[v] = g;
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
    n_pass += __shfl_xor_sync(0xffffffffu, n_pass, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_eval) atomicAdd(&head->n_eval, n_eval);
    if (n_pass) atomicAdd(&head->n_pass, n_pass);
  }
}

}  // namespace

cudaError_t launch_gamma(const double* ref, const double* ev, int nx, int ny, int nz, void* plan, double dose_pct,
                         double threshold, float* gamma, cudaStream_t s) {
  // queried once per process (a function-local static is initialised exactly once, also when
  // several host threads arrive together)
  struct Shape {
    cudaError_t e;
    int n_sm, occ[2];
  };
  static const Shape sh = [] {
    Shape r{cudaSuccess, 0, {0, 0}};
    int dev = 0;
    r.e = cudaGetDevice(&dev);
    if (r.e == cudaSuccess) r.e = cudaDeviceGetAttribute(&r.n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (r.e == cudaSuccess) r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ[0], dose_max_kernel, 256, 0);
    if (r.e == cudaSuccess) r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ[1], gamma_kernel, 256, 0);
    return r;
  }();
  if (sh.e != cudaSuccess) return sh.e;
  const int n_sm = sh.n_sm;
  const int* occ = sh.occ;
  GammaHead* head = static_cast<GammaHead*>(plan);
  const GammaOffset* off = reinterpret_cast<const GammaOffset*>(static_cast<unsigned char*>(plan) + kGammaHeadBytes);
  const long long n = static_cast<long long>(nx) * ny * nz;
  const bool vec = (reinterpret_cast<uintptr_t>(ref) & 15u) == 0 && (reinterpret_cast<uintptr_t>(gamma) & 15u) == 0;
  cudaError_t e = cudaMemsetAsync(head, 0, offsetof(GammaHead, n_off), s);
  if (e != cudaSuccess) return e;
  const long long units = ((vec ? n / 4 : n) + 255) / 256;
  auto grid_for = [&](int o) {
    const long long cap = static_cast<long long>(n_sm) * (o > 0 ? o : 1);
    return static_cast<int>(units < 1 ? 1 : (units < cap ? units : cap));
  };
  dose_max_kernel<<<grid_for(occ[0]), 256, 0, s>>>(ref, n, vec, head);
  gamma_kernel<<<grid_for(occ[1]), 256, 0, s>>>(ref, ev, nx, ny, nz, vec, head, off, dose_pct, threshold, gamma);
  return cudaGetLastError();
}

}  // namespace pmc
