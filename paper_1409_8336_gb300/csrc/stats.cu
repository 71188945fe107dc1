// stats.cu -- dose statistics (Sec. II.B.2: total and RMS dose per voxel from the
// group tallies) and the device-side single-routine checks used by the tests.
#include "pmc_kernels.cuh"

namespace pmc {
namespace {

// One thread per voxel: the voxel's group tallies are contiguous ([voxel][group]),
// so a warp streams 32 consecutive voxels' tallies through the same cache lines.
__global__ void __launch_bounds__(256) stats_kernel(const StatsArgs a) {
  const long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  __shared__ Physics ph_s;
  {
    const int4* src = reinterpret_cast<const int4*>(a.phys);
    int4* dst = reinterpret_cast<int4*>(&ph_s);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(Physics) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (v >= a.n_vox) return;
  const long long* t = reinterpret_cast<const long long*>(a.tally) + v * a.B;
  double s = 0.0;
  for (int b = 0; b < a.B; ++b) s += static_cast<double>(t[b]);
  const double mean = s / a.B;
  double ss = 0.0;
  for (int b = 0; b < a.B; ++b) {
    const double d = static_cast<double>(t[b]) - mean;
    ss += d * d;
  }
  int m;
  float rho;
  voxel_props(ph_s, a.g, static_cast<int>(v), m, rho);
  // MeV (2^-24 units) -> Gy: E * 1.602176634e-13 J / (rho * V * 1e-3 kg)
  const double vol = static_cast<double>(a.g.dx) * a.g.dy * a.g.dz;
  const double scale = rho > 0.0f ? (1.602176634e-10 / (static_cast<double>(rho) * vol)) / kFixD : 0.0;
  a.dose[v] = s * scale;
  a.sigma[v] = a.B > 1 ? sqrt(static_cast<double>(a.B) / (a.B - 1) * ss) * scale : 0.0;
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
  const long long blocks = (a.n_vox + 255) / 256;
  stats_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(a);
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
