// stats.cu -- dose statistics (Sec. II.B.2: total and RMS dose per voxel from the
// group tallies) and the device-side single-routine checks used by the tests.
#include "pmc_kernels.cuh"

namespace pmc {
namespace {

// int64 -> float without a 64-bit conversion instruction (those run on the
// narrow FP64 pipe): split into a signed high part and a 24-bit low part.
__device__ __forceinline__ float ll2f(long long x) {
  return static_cast<float>(static_cast<int>(x >> 24)) * 16777216.0f + static_cast<float>(static_cast<int>(x & 0xFFFFFF));
}

// One thread per voxel (grid-stride): the voxel's group tallies are contiguous
// ([voxel][group]), so a warp streams 32 consecutive voxels' tallies through the
// same cache lines.  The total is an exact integer sum; the spread is computed
// from single-precision deviations from the first group (a statistical estimate
// needs no more), so only the two outputs touch the FP64 pipe.
__global__ void __launch_bounds__(256) stats_kernel(const StatsArgs a) {
  const double vol = static_cast<double>(a.g.dx) * a.g.dy * a.g.dz;
  const float inv_b = 1.0f / static_cast<float>(a.B);
  const float corr = a.B > 1 ? static_cast<float>(a.B) / static_cast<float>(a.B - 1) : 0.0f;
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < a.n_vox;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long* t = reinterpret_cast<const long long*>(a.tally) + v * a.B;
    const long long t0 = t[0];
    long long sum = 0;
    float s1 = 0.0f, s2 = 0.0f;
    for (int b = 0; b < a.B; ++b) {
      const long long x = t[b];
      sum += x;
      const float d = ll2f(x - t0);
      s1 += d;
      s2 = fmaf(d, d, s2);
    }
    // sum over groups of (D_b - mean)^2 = s2 - s1^2 / B, with deviations from group 0
    const float ss = fmaxf(s2 - s1 * s1 * inv_b, 0.0f);
    int m;
    float rho;
    voxel_props(*a.phys, a.g, static_cast<int>(v), m, rho);
    // MeV (2^-24 units) -> Gy: E * 1.602176634e-13 J / (rho * V * 1e-3 kg).  1 / (rho V) from
    // a single-precision reciprocal refined by one Newton step in double (relative error
    // ~1e-14): a double division would take a dozen instructions of the narrow FP64 pipe per
    // voxel, which bound this kernel.
    double scale = 0.0;
    if (rho > 0.0f) {
      const double rv = static_cast<double>(rho) * vol;
      double r = static_cast<double>(__frcp_rn(static_cast<float>(rv)));
      r = r * fma(-rv, r, 2.0);
      scale = (1.602176634e-10 / kFixD) * r;
    }
    a.dose[v] = static_cast<double>(sum) * scale;
    a.sigma[v] = static_cast<double>(sqrtf(corr * ss)) * scale;
    if (a.let_num) {
      // LET_d = sum num / sum den; its standard error by the ratio estimator over the
      // groups: var = B/(B-1) sum_b (num_b - LET_d den_b)^2 / den^2
      const long long* tn = reinterpret_cast<const long long*>(a.let_num) + v * a.B;
      const long long* td = reinterpret_cast<const long long*>(a.let_den) + v * a.B;
      long long sn = 0, sd = 0;
      for (int b = 0; b < a.B; ++b) {
        sn += tn[b];
        sd += td[b];
      }
      if (sd > 0) {
        const double let = static_cast<double>(sn) / static_cast<double>(sd);
        const float lf = static_cast<float>(let);
        float e2 = 0.0f;
        for (int b = 0; b < a.B; ++b) {
          const float e = ll2f(tn[b]) - lf * ll2f(td[b]);
          e2 = fmaf(e, e, e2);
        }
        a.let[v] = let;
        a.let_sigma[v] = static_cast<double>(sqrtf(corr * e2) / ll2f(sd));
      } else {
        a.let[v] = 0.0;
        a.let_sigma[v] = 0.0;
      }
    }
  }
}

__global__ void debug_philox_kernel(const uint4* ctr, uint2 key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

__global__ void debug_tables_kernel(const Physics* ph, const float2* rt, const float2* et, int cls, const double* E,
                                    double* r, double* e, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float Ef = static_cast<float>(E[i]);
  const float R = range_mass(*ph, rt, cls, Ef, logf(Ef));
  r[i] = R;
  e[i] = energy_of_range(*ph, et, cls, R);
}

__global__ void debug_elastic_kernel(const Physics* ph, int nuclide, float E, const double* u, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ElasticOut o = elastic_kinematics(ph->nuc[nuclide], E, static_cast<float>(u[3 * i]),
                                          static_cast<float>(u[3 * i + 1]));
  double* d = out + 5ull * i;
  d[0] = o.T1; d[1] = o.c1; d[2] = o.T2; d[3] = o.c2; d[4] = o.ccm;
}

}  // namespace

cudaError_t launch_stats(const StatsArgs& a, cudaStream_t s) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const long long need = (a.n_vox + 255) / 256;
  const long long blocks = need < 8ll * n_sm ? need : 8ll * n_sm;
  stats_kernel<<<static_cast<unsigned>(blocks > 0 ? blocks : 1), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint4* ctr, uint2 key, uint4* out, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  debug_philox_kernel<<<(n + 255) / 256, 256, 0, s>>>(ctr, key, out, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_tables(const Physics* ph, const float2* rt, const float2* et, int cls, const double* E,
                                double* r, double* e, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  debug_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(ph, rt, et, cls, E, r, e, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_elastic(const Physics* ph, int nuclide, float E, const double* u, double* out, int n,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  debug_elastic_kernel<<<(n + 255) / 256, 256, 0, s>>>(ph, nuclide, E, u, out, n);
  return cudaGetLastError();
}

}  // namespace pmc
