// cascade.cu -- the non-elastic event generator's kernels (Sec. II.A.4): the cascade of a
// generation's queued events (persistent, one event per lane with refill), the evaporation
// of their residual nuclei (tiles sorted by mass number and excitation so that a warp's
// chains are alike), the event generator on its own (Table I workload), the debug entry and
// the event summaries that train the learned stand-in.  The physics is in cascade_event.cuh.
#include "cascade_event.cuh"

namespace pmc {
namespace {

__device__ __forceinline__ void stage_tables(const CascadeArgs& a, NucleusModel* nuc, float* bt) {
  const float* src = reinterpret_cast<const float*>(a.nuclei);
  float* dst = reinterpret_cast<float*>(nuc);
  const int nw = a.n_nuc * static_cast<int>(sizeof(NucleusModel) / 4);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
  for (int i = threadIdx.x; i < kBtabFloats; i += blockDim.x) bt[i] = a.btab[i];
  __syncthreads();
}

// Cascade stage: persistent; each lane runs one event at a time, one flight per
// iteration of a single loop, and takes the next event from the queue as soon as
// its own is done (warp-aggregated claims), so lanes do not wait at loop exits
// for the longest cascade of the warp.  A finished cascade emits its escaping
// nucleons and leaves its residual nucleus, with the position of its random
// stream, for the evaporation kernel.
// Resident blocks: the primaries' ~1.2e5 events take one or two per lane, so more lanes shorten
// the launch while the registers stay spill-free: 4 blocks of 128 (117 registers) for the
// cascade, 7 (72) for the evaporation, whose ~940 tiles then fit one wave (uncapped: 153 and 156
// registers, 3 blocks per SM; slab step 5.37 -> 5.28 ms; 6 cascade blocks spill, 1.08 ms).
__global__ void __launch_bounds__(128, 4) inc_kernel(const CascadeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned n = min(*a.qne_count, a.qne_cap);
  if (n == 0) return;
  NucleusModel* nuc = reinterpret_cast<NucleusModel*>(smem);
  float* bt = reinterpret_cast<float*>(nuc + a.n_nuc);
  stage_tables(a, nuc, bt);
  const unsigned long long seed = *a.seed;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  const unsigned lane = threadIdx.x & 31u;
  TransportSink sk;
  sk.env.a = &a;
  sk.key = key;
  sk.dep = sk.esc = sk.bnd = 0;
  sk.sec = sk.dropped = sk.retries = sk.n_transparent = 0;
  IncP P[kIncStack];
  IncState s;
  Stream st{key, 0ull, 0u, 4, make_float4(0.f, 0.f, 0.f, 0.f)};
  const NucleusModel* nu = nuc;
  bool have = false, drained = false, setup = false;
  int attempt = 0, retries = 0;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !have && !drained);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned base = 0;
      if (static_cast<int>(lane) == leader) base = atomicAdd(a.work, static_cast<unsigned>(__popc(need)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!have && !drained) {
        const unsigned idx = base + __popc(need & ((1u << lane) - 1u));
        if (idx < n) {
          sk.ev = a.qne[idx];
          sk.b = sk.ev.root % static_cast<unsigned>(a.B);
          st = Stream{key, sk.ev.pid, 0u, 4, make_float4(0.f, 0.f, 0.f, 0.f)};
          nu = nuc + sk.ev.target;
          attempt = 0;
          retries = 0;
          setup = true;
          have = true;
        } else {
          drained = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, !have && drained)) break;
    if (!have) continue;
    if (setup) {
      inc_setup(*nu, sk.ev.E, st, P, s);
      setup = false;
      continue;
    }
    if (!inc_flight(*nu, st, P, s)) continue;
    P[s.ip] = s.p;
    if (++s.ip < s.n) {
      s.p = P[s.ip];
      s.crossings = 0;
      s.iters = 0;
      continue;
    }
    Residual r;
    if (!inc_residual(*nu, bt, sk.ev.E, P, s, r)) {
      ++retries;
      if (++attempt < kIncRetries) {
        setup = true;
      } else {
        sk.transparent(retries);
        have = false;
      }
      continue;
    }
    const int k = inc_emit(P, s.n, sk);
    const unsigned ri = atomicAdd(a.rec_count, 1u);
    if (ri < a.rec_cap) {
      EvapRecord& e = a.rec[ri];
      e.ev = sk.ev;
      e.Ex = r.Ex; e.px = r.px; e.py = r.py; e.pz = r.pz; e.bind = r.bind;
      e.buf = st.buf; e.draw = st.draw; e.pos = st.pos;
      e.Z = r.Z; e.A = r.A; e.k = k; e.retries = retries;
    } else {
      evaporate(bt, st, r, k, retries, sk);   // no room to hand it on (cannot happen: one record per event)
    }
    have = false;
  }
  flush_counters(sk, a.cnt);
}

// Evaporation stage: one residual per thread; each block sorts its tile of 128
// residuals by (mass number, excitation) so that a warp's chains are alike.
__global__ void __launch_bounds__(128, 7) evap_kernel(const CascadeArgs a) {
  __shared__ float bt[kBtabFloats];
  __shared__ unsigned long long keys[128];
  const unsigned n = min(*a.rec_count, a.rec_cap);
  if (n == 0 || blockIdx.x * blockDim.x >= n) return;
  for (int i = threadIdx.x; i < kBtabFloats; i += blockDim.x) bt[i] = a.btab[i];
  __syncthreads();
  const unsigned long long seed = *a.seed;
  TransportSink sk;
  sk.env.a = &a;
  sk.key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  sk.dep = sk.esc = sk.bnd = 0;
  sk.sec = sk.dropped = sk.retries = sk.n_transparent = 0;
  for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned i = base + threadIdx.x;
    unsigned long long key = ~0ull;
    if (i < n) {
      const EvapRecord& e = a.rec[i];
      const float ex = static_cast<float>(fmax(e.Ex, 0.0));
      key = (static_cast<unsigned long long>(e.A) << 56) | (static_cast<unsigned long long>(__float_as_uint(ex)) << 24) |
            threadIdx.x;
    }
    keys[threadIdx.x] = key;
    __syncthreads();
    for (unsigned kk = 2; kk <= 128; kk <<= 1) {          // bitonic sort of the tile
      for (unsigned j = kk >> 1; j > 0; j >>= 1) {
        const unsigned t = threadIdx.x, l = t ^ j;
        if (l > t) {
          const unsigned long long x = keys[t], y = keys[l];
          const bool up = (t & kk) == 0;
          if ((x > y) == up) { keys[t] = y; keys[l] = x; }
        }
        __syncthreads();
      }
    }
    const unsigned long long mine = keys[threadIdx.x];
    __syncthreads();
    if (mine != ~0ull) {
      const EvapRecord& e = a.rec[base + static_cast<unsigned>(mine & 0xFFu)];
      sk.ev = e.ev;
      sk.b = sk.ev.root % static_cast<unsigned>(a.B);
      Stream st{sk.key, e.ev.pid, e.draw, e.pos, e.buf};
      Residual r;
      r.Ex = e.Ex; r.px = e.px; r.py = e.py; r.pz = e.pz; r.bind = e.bind; r.Z = e.Z; r.A = e.A;
      evaporate(bt, st, r, e.k, e.retries, sk);
    }
  }
  flush_counters(sk, a.cnt);
}

// Sink of the debug entry point: products written as rows.
struct TableSink {
  double* summary;
  double* products;
  int cap, n;
  __device__ void product(int k, int species, double T, float ax, float ay, float az) {
    if (k < cap) {
      double* o = products + static_cast<size_t>(k) * 5;
      o[0] = species; o[1] = T; o[2] = ax; o[3] = ay; o[4] = az;
    }
    n = k + 1;
  }
  __device__ void residual(int Z, int A, double Tres, double Ex, double bind, int r) {
    summary[0] = n; summary[1] = Z; summary[2] = A; summary[3] = Tres; summary[4] = Ex;
    summary[5] = bind; summary[6] = r; summary[7] = 0;
  }
  __device__ void transparent(int r) {
    summary[0] = 0; summary[6] = r; summary[7] = 1;
  }
};

__global__ void debug_inc_kernel(const NucleusModel* nu, const float* bt, float E, unsigned long long seed,
                                 unsigned long long pid0, int n, double* summary, double* products, int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  IncP P[kIncStack];
  TableSink sk{summary + 8ull * i, products + 5ull * cap * i, cap, 0};
  nonelastic_event(*nu, bt, E, make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32)),
                   pid0 + i, P, sk);
}

// Sink of the event-generator entry point: per-thread yields of the events it runs.
struct YieldSink {
  unsigned long long n_transparent, retries, count[6];
  long long energy[6], res, ex, bind;
  __device__ void product(int, int species, double T, float, float, float) {
    ++count[species];
    energy[species] += fixd(T);
  }
  __device__ void residual(int, int, double Tres, double Ex, double b, int r) {
    res += fixd(Tres);
    ex += fixd(Ex);
    bind += fixd(b);
    retries += r;
  }
  __device__ void transparent(int r) {
    retries += r;
    ++n_transparent;
  }
};

// n non-elastic events of a proton of energy E on one nucleus (Sec. II.A.4), one
// event per thread, event i with the random stream of particle pid0 + i.  Yields are
// reduced per warp and added to `out` as integers (energies in 2^-24 MeV), so the
// totals do not depend on the order of the events.
__global__ void __launch_bounds__(128) inc_yield_kernel(const NucleusModel* __restrict__ nu,
                                                        const float* __restrict__ btab, float E,
                                                        unsigned long long seed, unsigned long long pid0,
                                                        unsigned long long n, EventYields* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  NucleusModel* nuc = reinterpret_cast<NucleusModel*>(smem);
  float* bt = reinterpret_cast<float*>(nuc + 1);
  {
    const float* src = reinterpret_cast<const float*>(nu);
    float* dst = reinterpret_cast<float*>(nuc);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(NucleusModel) / 4); i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < kBtabFloats; i += blockDim.x) bt[i] = btab[i];
  }
  __syncthreads();
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  YieldSink sk{};
  unsigned long long events = 0;
  IncP P[kIncStack];
  for (unsigned long long i = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    nonelastic_event(*nuc, bt, E, key, pid0 + i, P, sk);
    ++events;
  }
  auto wsum = [](unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  auto add = [&](unsigned long long* dst, unsigned long long x) {
    x = wsum(x);
    if ((threadIdx.x & 31u) == 0 && x) atomicAdd(dst, x);
  };
  add(&out->events, events);
  add(&out->transparent, sk.n_transparent);
  add(&out->retries, sk.retries);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    add(&out->count[k], sk.count[k]);
    add(reinterpret_cast<unsigned long long*>(&out->energy[k]), static_cast<unsigned long long>(sk.energy[k]));
  }
  add(reinterpret_cast<unsigned long long*>(&out->residual), static_cast<unsigned long long>(sk.res));
  add(reinterpret_cast<unsigned long long*>(&out->excitation), static_cast<unsigned long long>(sk.ex));
  add(reinterpret_cast<unsigned long long*>(&out->binding), static_cast<unsigned long long>(sk.bind));
}

}  // namespace

// SM count and resident blocks per SM of a persistent launch, with the query's status.
struct LaunchShape {
  cudaError_t e;
  int n_sm, bps;
};

cudaError_t launch_inc_yields(const NucleusModel* nu, const float* btab, float E, unsigned long long seed,
                              unsigned long long pid0, unsigned long long n, EventYields* out, cudaStream_t s) {
  const size_t smem = sizeof(NucleusModel) + kBtabFloats * sizeof(float);
  // queried once per process (a function-local static is initialised exactly once, also
  // when several host threads arrive together)
  static const LaunchShape sh = [smem] {
    LaunchShape r{cudaSuccess, 0, 0};
    int dev = 0;
    r.e = cudaGetDevice(&dev);
    if (r.e == cudaSuccess) r.e = cudaDeviceGetAttribute(&r.n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (r.e == cudaSuccess) r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.bps, inc_yield_kernel, 128, smem);
    return r;
  }();
  if (sh.e != cudaSuccess) return sh.e;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(EventYields), s);
  if (e != cudaSuccess || n == 0) return e;
  const unsigned long long want = (n + 127) / 128;
  const unsigned long long cap = static_cast<unsigned long long>(sh.n_sm) * (sh.bps > 0 ? sh.bps : 1);
  inc_yield_kernel<<<static_cast<unsigned>(want < cap ? want : cap), 128, smem, s>>>(nu, btab, E, seed, pid0, n, out);
  return cudaGetLastError();
}

cudaError_t launch_cascade(const CascadeArgs& a, cudaStream_t s) {
  const size_t smem = a.n_nuc * sizeof(NucleusModel) + kBtabFloats * sizeof(float);
  // queried once per process, for the largest table (the multi-plan stream's slot threads
  // may arrive together: a function-local static is initialised exactly once)
  static const LaunchShape sh = [] {
    LaunchShape r{cudaSuccess, 0, 0};
    int dev = 0;
    r.e = cudaGetDevice(&dev);
    if (r.e == cudaSuccess) r.e = cudaDeviceGetAttribute(&r.n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (r.e == cudaSuccess)
      r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.bps, inc_kernel, 128,
                                                          kMaxNuc * sizeof(NucleusModel) + kBtabFloats * sizeof(float));
    if (r.bps < 1) r.bps = 1;
    return r;
  }();
  if (sh.e != cudaSuccess) return sh.e;
  inc_kernel<<<sh.n_sm * sh.bps, 128, smem, s>>>(a);
  evap_kernel<<<sh.n_sm * 8, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_debug_inc(const NucleusModel* nu, const float* btab, float E, unsigned long long seed,
                             unsigned long long pid0, int n, double* summary, double* products, int cap,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  debug_inc_kernel<<<(n + 127) / 128, 128, 0, s>>>(nu, btab, E, seed, pid0, n, summary, products, cap);
  return cudaGetLastError();
}

}  // namespace pmc

// ---------------------------------------------------------------------------
// Event summaries for training the learned stand-in of the event generator
// (the paper has no counterpart).  Row per event, in the frame where the
// incident proton moves along +z: E, target slot, number of protons above
// E_cut, their kinetic energies / E and polar cosines for the four most
// energetic (zero-padded), and the locally deposited energy / E (fragments
// heavier than protons, the residual recoil, protons below E_cut and protons
// beyond the fourth).
// ---------------------------------------------------------------------------
namespace pmc {
namespace {

struct SummarySink {
  float E;
  int np;
  float T[kSurrSlots], c[kSurrSlots];
  double local;
  __device__ void product(int, int species, double T_, float, float, float az) {
    const float t = static_cast<float>(T_);
    if (species == 1 && t > kEcut) {
      ++np;
      // keep the kSurrSlots most energetic, sorted descending
      float tv = t, cv = az;
      for (int k = 0; k < kSurrSlots; ++k) {
        if (tv > T[k]) {
          const float ot = T[k], oc = c[k];
          T[k] = tv; c[k] = cv; tv = ot; cv = oc;
        }
      }
      local += tv;   // the displaced (or rejected) fifth proton deposits locally
    } else if (species != 0) {
      local += T_;
    }
  }
  __device__ void residual(int, int, double Tres, double, double, int) { local += Tres; }
  __device__ void transparent(int) { np = -1; }
};

__global__ void surrogate_dataset_kernel(const NucleusModel* nuclei, const float* bt, const int* slot_nuc, int n_slots,
                                         unsigned long long seed, unsigned long long n, float* out) {
  const unsigned long long i = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  // energy uniform in [10, 250] MeV and a target slot, from the event's own stream (tag 6)
  const float4 u = draw4(key, i, 0u, 6u);
  const float E = 10.0f + 240.0f * u.x;
  const int slot = min(static_cast<int>(u.y * n_slots), n_slots - 1);
  IncP P[kIncStack];
  SummarySink sk;
  sk.E = E;
  sk.np = 0;
  sk.local = 0.0;
  for (int k = 0; k < kSurrSlots; ++k) { sk.T[k] = 0.0f; sk.c[k] = 0.0f; }
  nonelastic_event(nuclei[slot_nuc[slot]], bt, E, key, i, P, sk);
  float* o = out + i * kSurrFeatures;
  o[0] = E;
  o[1] = static_cast<float>(slot);
  o[2] = static_cast<float>(sk.np);
  for (int k = 0; k < kSurrSlots; ++k) {
    o[3 + k] = sk.T[k] / E;
    o[3 + kSurrSlots + k] = sk.c[k];
  }
  o[3 + 2 * kSurrSlots] = static_cast<float>(sk.local / E);
}

}  // namespace

cudaError_t launch_surrogate_dataset(const NucleusModel* nuclei, const float* btab, const int* slot_nuc, int n_slots,
                                     unsigned long long seed, unsigned long long n, float* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  surrogate_dataset_kernel<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(nuclei, btab, slot_nuc, n_slots,
                                                                                   seed, n, out);
  return cudaGetLastError();
}

}  // namespace pmc
