// surrogate.cu -- a learned stand-in for the intranuclear-cascade + evaporation
// event generator (the paper has no counterpart; its event generator is the
// reference this network is trained on and judged against).
//
// A conditional quantile network: an MLP 32-256-256-256-256-16 with ReLU,
// trained with the pinball loss, maps (incident energy, target, a multiplicity
// token, ten uniforms) to quantiles of the event's summary: the number of
// protons above E_cut, the energies and polar cosines of up to four of them,
// and the locally deposited energy.  Inference runs it twice per event: once
// with the token "unknown" for the multiplicity, then with the sampled
// multiplicity for the rest.
//
// Dense layers run on the tensor cores: BF16 operands (weights and activations
// rounded from FP32 master copies when a tile is staged in shared memory), FP32
// accumulation, with the warp-level mma.sync m16n8k16 instruction.
#include <cuda_bf16.h>

#include "pmc_kernels.cuh"

namespace pmc {
namespace {

constexpr int kTileM = 64, kTileN = 64, kTileK = 32, kPad = 8;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] (=|+=) sum_k A(m,k) B(k,n) (+ bias[n]) (ReLU) (* [mask[m][n] > 0]).
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]; FP32 in memory, BF16 math.
// The row count is *Mp when Mp is given (device-resident), else M.
__global__ void __launch_bounds__(128) gemm_kernel(int M, const unsigned* Mp, int N, int K, const float* __restrict__ A,
                                                   long long sam, long long sak, const float* __restrict__ B,
                                                   long long sbk, long long sbn, float* __restrict__ C, long long ldc,
                                                   const float* __restrict__ bias, int relu,
                                                   const float* __restrict__ mask, int accumulate) {
  const int rows = Mp ? static_cast<int>(min(*Mp, static_cast<unsigned>(M))) : M;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * kTileN;
  if (m0 >= rows) return;
  __shared__ __nv_bfloat16 As[kTileM][kTileK + kPad];
  __shared__ __nv_bfloat16 Bs[kTileN][kTileK + kPad];   // stored [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // warp's 32x32 sub-tile
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += kTileK) {
    for (int e = tid; e < kTileM * kTileK; e += 128) {
      const int mm = e / kTileK, kk = e % kTileK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[mm][kk] = __float2bfloat16_rn(gm < rows && gk < K ? A[gm * sam + gk * sak] : 0.0f);
    }
    for (int e = tid; e < kTileN * kTileK; e += 128) {
      const int nn = e / kTileK, kk = e % kTileK;
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[nn][kk] = __float2bfloat16_rn(gn < N && gk < K ? B[gk * sbk + gn * sbn] : 0.0f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; kk += 16) {
      unsigned af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        const int c = kk + 2 * t;
        af[i][0] = pack_bf16(__bfloat162float(As[r][c]), __bfloat162float(As[r][c + 1]));
        af[i][1] = pack_bf16(__bfloat162float(As[r + 8][c]), __bfloat162float(As[r + 8][c + 1]));
        af[i][2] = pack_bf16(__bfloat162float(As[r][c + 8]), __bfloat162float(As[r][c + 9]));
        af[i][3] = pack_bf16(__bfloat162float(As[r + 8][c + 8]), __bfloat162float(As[r + 8][c + 9]));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + 8 * j + g;
        const int c = kk + 2 * t;
        bfr[j][0] = pack_bf16(__bfloat162float(Bs[n][c]), __bfloat162float(Bs[n][c + 1]));
        bfr[j][1] = pack_bf16(__bfloat162float(Bs[n][c + 8]), __bfloat162float(Bs[n][c + 9]));
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * t + (r & 1);
        if (m >= rows || n >= N) continue;
        float v = acc[i][j][r];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.0f);
        if (mask && !(mask[static_cast<long long>(m) * ldc + n] > 0.0f)) v = 0.0f;
        float* dst = C + static_cast<long long>(m) * ldc + n;
        *dst = accumulate ? *dst + v : v;
      }
    }
  }
}

// Pinball loss of quantile predictions yhat against targets y at levels tau, per
// masked entry; gradient w.r.t. yhat scaled by 1/rows.
__global__ void pinball_kernel(int rows, const float* yhat, const float* y, const float* tau, const float* mask,
                               float* grad, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < rows * kSurrOut) {
    const float m = mask[i];
    const float u = y[i] - yhat[i];
    const float tq = tau[i];
    l = m * u * (tq - (u < 0.0f ? 1.0f : 0.0f));
    grad[i] = -m * (tq - (u < 0.0f ? 1.0f : 0.0f)) / static_cast<float>(rows);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / static_cast<float>(rows));
}

// Column sums (bias gradients): db[n] = sum_m G[m][n].
__global__ void colsum_kernel(int rows, int N, const float* G, float* db) {
  const int n = blockIdx.x;
  float s = 0.0f;
  for (int m = threadIdx.x; m < rows; m += blockDim.x) s += G[static_cast<long long>(m) * N + n];
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[n] = red[0];
}

// AdamW on the flat parameter vector.
__global__ void adamw_kernel(int n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                             float eps, float wd, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
}

// Training rows from event summaries: two rows per event.  Row 2i asks for the
// multiplicity (token -1); row 2i+1 gives the event's multiplicity and asks for
// the rest.  Uniforms from Philox keyed by (seed, step, row).
__global__ void train_rows_kernel(int batch, const float* feat, const unsigned* perm, unsigned long long first,
                                  unsigned long long n_events, unsigned long long seed, unsigned step, float* X,
                                  float* Y, float* tau, float* mask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * batch) return;
  const unsigned long long ev = perm[(first + r / 2) % n_events];
  const float* f = feat + ev * kSurrFeatures;
  const bool ask_np = (r & 1) == 0;
  const int np = min(static_cast<int>(f[2]), kSurrSlots);
  float* x = X + static_cast<long long>(r) * kSurrIn;
  float* y = Y + static_cast<long long>(r) * kSurrOut;
  float* tq = tau + static_cast<long long>(r) * kSurrOut;
  float* mk = mask + static_cast<long long>(r) * kSurrOut;
  for (int j = 0; j < kSurrIn; ++j) x[j] = 0.0f;
  x[0] = (f[0] - 130.0f) / 120.0f;
  x[1 + static_cast<int>(f[1])] = 1.0f;
  x[1 + kSurrTargets] = ask_np ? -1.0f : static_cast<float>(np) / kSurrSlots;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  float u[12];
  const float4 u0 = draw4(key, (static_cast<unsigned long long>(step) << 32) | r, 0u, 7u);
  const float4 u1 = draw4(key, (static_cast<unsigned long long>(step) << 32) | r, 1u, 7u);
  const float4 u2 = draw4(key, (static_cast<unsigned long long>(step) << 32) | r, 2u, 7u);
  u[0] = u0.x; u[1] = u0.y; u[2] = u0.z; u[3] = u0.w; u[4] = u1.x; u[5] = u1.y;
  u[6] = u1.z; u[7] = u1.w; u[8] = u2.x; u[9] = u2.y; u[10] = u2.z; u[11] = u2.w;
  for (int j = 0; j < kSurrTau; ++j) x[2 + kSurrTargets + j] = u[j];
  for (int j = 0; j < kSurrOut; ++j) { y[j] = 0.0f; tq[j] = 0.5f; mk[j] = 0.0f; }
  if (ask_np) {
    y[0] = static_cast<float>(np);
    tq[0] = u[0];
    mk[0] = 1.0f;
  } else {
    for (int k = 0; k < kSurrSlots; ++k) {
      y[1 + k] = f[3 + k];
      tq[1 + k] = u[1 + k];
      mk[1 + k] = k < np ? 1.0f : 0.0f;
      y[1 + kSurrSlots + k] = f[3 + kSurrSlots + k];
      tq[1 + kSurrSlots + k] = u[1 + kSurrSlots + k];
      mk[1 + kSurrSlots + k] = k < np ? 1.0f : 0.0f;
    }
    y[1 + 2 * kSurrSlots] = f[3 + 2 * kSurrSlots];
    tq[1 + 2 * kSurrSlots] = u[1 + 2 * kSurrSlots];
    mk[1 + 2 * kSurrSlots] = 1.0f;
  }
}

// Inference row of a queued event: energy, target one-hot, multiplicity token
// (-1 in the first pass) and ten uniforms from the event's own stream (tag 8).
__device__ void event_row(const Particle& ev, const int* nuc_slot, uint2 key, float* x) {
  for (int j = 0; j < kSurrIn; ++j) x[j] = 0.0f;
  x[0] = (ev.E - 130.0f) / 120.0f;
  x[1 + nuc_slot[ev.target]] = 1.0f;
  x[1 + kSurrTargets] = -1.0f;
  const float4 u0 = draw4(key, ev.pid, 0u, 8u), u1 = draw4(key, ev.pid, 1u, 8u), u2 = draw4(key, ev.pid, 2u, 8u);
  const float u[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
  for (int j = 0; j < kSurrTau; ++j) x[2 + kSurrTargets + j] = u[j];
}

__device__ __forceinline__ int multiplicity(float q) {
  return min(max(static_cast<int>(floorf(q + 0.5f)), 0), kSurrSlots);
}

// Emits an event from the network's quantiles: protons to the secondary queue,
// the local deposit to the event voxel, the rest (neutrons, photons, binding)
// escapes.  Energy is conserved by construction.
__device__ void emit_event(const Particle& ev, const float* y1, const float* y2, uint2 key, unsigned long long* tally,
                           int B, Particle* qsec, unsigned* qsec_count, unsigned qsec_cap, long long* hist,
                           unsigned long long hist_n, long long& dep, long long& esc, unsigned long long& sec,
                           unsigned long long& dropped) {
  const int np = multiplicity(y1[0]);
  float T[kSurrSlots], c[kSurrSlots];
  float sum = 0.0f;
  for (int k = 0; k < kSurrSlots; ++k) {
    T[k] = k < np ? fmaxf(y2[1 + k], 0.0f) * ev.E : 0.0f;
    c[k] = fminf(fmaxf(y2[1 + kSurrSlots + k], -1.0f), 1.0f);
    sum += T[k];
  }
  float loc = fmaxf(y2[1 + 2 * kSurrSlots], 0.0f) * ev.E;
  sum += loc;
  if (sum > ev.E) {                                // never more energy out than in
    const float sc = ev.E / sum;
    for (int k = 0; k < kSurrSlots; ++k) T[k] *= sc;
    loc *= sc;
  }
  const unsigned b = ev.root % static_cast<unsigned>(B);
  const float4 ua = draw4(key, ev.pid, 3u, 8u);
  const float uphi[4] = {ua.x, ua.y, ua.z, ua.w};
  long long handed = 0;
  for (int k = 0; k < np; ++k) {
    if (T[k] <= kEcut) { loc += T[k]; continue; }
    float sp, cp;
    sincospif(2.0f * uphi[k], &sp, &cp);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - c[k] * c[k]));
    const float3 d = frame_to_lab(ev.u, ev.v, ev.w, st * cp, st * sp, c[k]);
    Particle r;
    r.x = ev.x; r.y = ev.y; r.z = ev.z; r.u = d.x; r.v = d.y; r.w = d.z; r.E = T[k];
    r.voxel = ev.voxel; r.pid = child_pid(key, ev.pid, static_cast<unsigned>(k)); r.root = ev.root; r.target = -1;
    const unsigned slot = atomicAdd(qsec_count, 1u);
    if (slot < qsec_cap) {
      qsec[slot] = r;
      ++sec;
      handed += fix(T[k]);
    } else {
      ++dropped;
      loc += T[k];
    }
  }
  const long long qE = fix(ev.E), ql = fix(loc);
  const long long qesc = qE - handed - ql;       // neutrons, photons and binding: leave the grid
  atomicAdd(tally + static_cast<size_t>(ev.voxel) * B + b, static_cast<unsigned long long>(ql));
  dep += ql;
  esc += qesc;
  if (hist && ev.root < hist_n) {
    atomicAdd(reinterpret_cast<unsigned long long*>(hist + 4ull * ev.root + 1), static_cast<unsigned long long>(ql));
    atomicAdd(reinterpret_cast<unsigned long long*>(hist + 4ull * ev.root + 2), static_cast<unsigned long long>(qesc));
  }
}

// Fused inference: one block takes 64 rows at a time (persistent over the
// device-resident row count), keeps their activations in shared memory as BF16
// through all five layers, and streams the layers' BF16 weights in 64x64
// chunks by cp.async (global -> shared, bypassing L1) through three buffers:
// the copies of the next two chunks, across layer boundaries, are in flight
// while the tensor cores consume the current one (FP32 accumulation).
// Two launches per generation replace ten layer GEMMs and their activations in
// global memory.
constexpr int kActLd = kSurrHidden + 8;          // padded row (conflict-free fragment loads)
constexpr int kChunk = 64;                       // k-chunk of streamed weights
constexpr int kWLd = kChunk + 8;                 // 144-byte rows, 16-byte aligned
constexpr int kWStages = 3;                      // weight-chunk buffers
constexpr int kInferSmem = 2 * 64 * kActLd * 2 + kWStages * 64 * kWLd * 2;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_newest_pending() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Position of the weight-chunk stream: layer l, chunk c of that layer (n-tile c / kpn,
// k-chunk c % kpn), and the layer's offset in the parameter vector.
struct ChunkCursor {
  int l = 0, c = 0;
  size_t off = 0;
};
__device__ __forceinline__ int layer_in(int l) { return l == 0 ? kSurrIn : kSurrHidden; }
__device__ __forceinline__ int layer_out(int l) { return l == kSurrLayers - 1 ? kSurrOut : kSurrHidden; }
__device__ __forceinline__ int layer_kc(int l) { return layer_in(l) < kChunk ? layer_in(l) : kChunk; }
__device__ __forceinline__ int layer_chunks(int l) { return (layer_out(l) + 63) / 64 * (layer_in(l) / layer_kc(l)); }

// Starts the copies of the cursor's chunk into buf (nothing past the last layer); rows of a
// chunk beyond the layer's outputs are zero-filled.
__device__ __forceinline__ void issue_chunk(const ChunkCursor& f, const __nv_bfloat16* __restrict__ Wb,
                                            __nv_bfloat16* buf) {
  if (f.l >= kSurrLayers) return;
  const int din = layer_in(f.l), dout = layer_out(f.l), kc = layer_kc(f.l), kpn = din / kc;
  const int n0 = (f.c / kpn) * 64, k0 = (f.c % kpn) * kc, vpr = kc / 8;
  const __nv_bfloat16* W = Wb + f.off;
  for (int v = threadIdx.x; v < 64 * vpr; v += blockDim.x) {
    const int nn = v / vpr, kv = (v % vpr) * 8;
    __nv_bfloat16* dst = buf + nn * kWLd + kv;
    if (n0 + nn < dout) cp_async16(dst, W + static_cast<size_t>(n0 + nn) * din + k0 + kv);
    else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
  }
}

__device__ __forceinline__ void advance_chunk(ChunkCursor& f) {
  if (f.l >= kSurrLayers) return;
  if (++f.c == layer_chunks(f.l)) {
    f.off += static_cast<size_t>(layer_in(f.l)) * layer_out(f.l) + layer_out(f.l);
    ++f.l;
    f.c = 0;
  }
}

// The five layers on one 64-row tile whose inputs are in the first activation buffer (columns
// 0..kSurrIn-1); the last layer's outputs for rows < nvalid go to out[r * kSurrOut + n].
__device__ __forceinline__ void mlp_tile(__nv_bfloat16* const tile, const __nv_bfloat16* __restrict__ Wb,
                         const float* __restrict__ P, float* out, int nvalid) {
  // shared memory of the tile: two activation buffers [64][kActLd], then kWStages weight
  // buffers [64][kWLd] (addressed arithmetically: no local-memory pointer arrays)
  __nv_bfloat16* const wbuf0 = tile + 2 * 64 * kActLd;
  auto wbuf = [&](int i) { return wbuf0 + i * (64 * kWLd); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  // prologue: the first two chunks in flight (one commit group per chunk, empty past the end)
  ChunkCursor f;
  issue_chunk(f, Wb, wbuf(0));
  cp_async_commit();
  advance_chunk(f);
  issue_chunk(f, Wb, wbuf(1));
  cp_async_commit();
  advance_chunk(f);
  size_t off = 0;
  int cur = 0, q = 0;
#pragma unroll 1
  for (int l = 0; l < kSurrLayers; ++l) {
    const int din = layer_in(l), dout = layer_out(l), kc = layer_kc(l), kpn = din / kc;
    const float* bias = P + off + static_cast<size_t>(din) * dout;
    const __nv_bfloat16* ain = tile + cur * (64 * kActLd);
    __nv_bfloat16* aout = tile + (cur ^ 1) * (64 * kActLd);
    const int n_chunks = layer_chunks(l);
    float acc[2][4][4];
#pragma unroll 1
    for (int c = 0; c < n_chunks; ++c, ++q) {
      const int n0 = (c / kpn) * 64, k0 = (c % kpn) * kc;
      cp_async_wait_newest_pending();   // this thread's copies of chunk q have landed
      __syncthreads();                  // everyone's have; chunk q-1 and the last epilogue are done
      issue_chunk(f, Wb, wbuf((q + 2) % kWStages));
      cp_async_commit();
      advance_chunk(f);
      if (c % kpn == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
      }
      const __nv_bfloat16* Ws = wbuf(q % kWStages);
      for (int kk = 0; kk < kc; kk += 16) {
        unsigned af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const __nv_bfloat16* a0 = ain + (wm + 16 * i + g) * kActLd + k0 + kk + 2 * t;
          af[i][0] = *reinterpret_cast<const unsigned*>(a0);
          af[i][1] = *reinterpret_cast<const unsigned*>(a0 + 8 * kActLd);
          af[i][2] = *reinterpret_cast<const unsigned*>(a0 + 8);
          af[i][3] = *reinterpret_cast<const unsigned*>(a0 + 8 * kActLd + 8);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat16* b0 = Ws + (wn + 8 * j + g) * kWLd + kk + 2 * t;
          bfr[j][0] = *reinterpret_cast<const unsigned*>(b0);
          bfr[j][1] = *reinterpret_cast<const unsigned*>(b0 + 8);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
      }
      if (c % kpn == kpn - 1) {                            // n-tile complete: epilogue
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
              const int r = wm + 16 * i + g + (r4 >= 2 ? 8 : 0);
              const int n = n0 + wn + 8 * j + 2 * t + (r4 & 1);
              if (n >= dout) continue;
              const float v = acc[i][j][r4] + bias[n];
              if (l < kSurrLayers - 1) {
                aout[r * kActLd + n] = __float2bfloat16_rn(fmaxf(v, 0.0f));
              } else if (r < nvalid) {
                out[r * kSurrOut + n] = v;
              }
            }
      }
    }
    off += static_cast<size_t>(din) * dout + dout;
    cur ^= 1;
  }
  __syncthreads();
}



// Rows X[n][kSurrIn] -> outputs Y[n][kSurrOut] (persistent over 64-row tiles).
__global__ void __launch_bounds__(128, 2) mlp_infer_kernel(const unsigned* n_rows, unsigned cap, const float* __restrict__ X,
                                                        const __nv_bfloat16* __restrict__ Wb,
                                                        const float* __restrict__ P, float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* const tile = reinterpret_cast<__nv_bfloat16*>(smem);   // act[0] = tile
  const unsigned rows = min(*n_rows, cap);
  for (unsigned r0 = blockIdx.x * 64u; r0 < rows; r0 += gridDim.x * 64u) {
    for (int e = threadIdx.x; e < 64 * kSurrIn; e += 128) {
      const int r = e / kSurrIn, c = e % kSurrIn;
      tile[r * kActLd + c] = __float2bfloat16_rn(r0 + r < rows ? X[static_cast<size_t>(r0 + r) * kSurrIn + c] : 0.0f);
    }
    mlp_tile(tile, Wb, P, Y + static_cast<size_t>(r0) * kSurrOut, static_cast<int>(min(64u, rows - r0)));
    __syncthreads();
  }
}

// The event stage of a generation with the learned stand-in, fused: per tile of 64
// queued events, build the inference rows, run the network (multiplicity pass),
// condition on the sampled multiplicity, run it again and emit the events, with rows
// and outputs in shared memory throughout.
constexpr int kEventSmem = kInferSmem + 64 * kSurrIn * 4 + 2 * 64 * kSurrOut * 4;

__global__ void __launch_bounds__(128, 2) surrogate_event_kernel(const unsigned* n_ev, unsigned cap,
                                                              const Particle* __restrict__ qne, const int* nuc_slot,
                                                              const unsigned long long* seedp,
                                                              const __nv_bfloat16* __restrict__ Wb,
                                                              const float* __restrict__ P, unsigned long long* tally,
                                                              int B, Particle* qsec, unsigned* qsec_count,
                                                              unsigned qsec_cap, Counters* cnt, long long* hist,
                                                              unsigned long long hist_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* const tile = reinterpret_cast<__nv_bfloat16*>(smem);   // act[0] = tile
  float* xin = reinterpret_cast<float*>(smem + kInferSmem);   // [64][kSurrIn]
  float* y1 = xin + 64 * kSurrIn;                              // [64][kSurrOut]
  float* y2 = y1 + 64 * kSurrOut;
  const unsigned rows = min(*n_ev, cap);
  const unsigned long long seed = *seedp;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  const int tid = threadIdx.x;
  long long dep = 0, esc = 0;
  unsigned long long sec = 0, dropped = 0;
  for (unsigned r0 = blockIdx.x * 64u; r0 < rows; r0 += gridDim.x * 64u) {
    const int nvalid = static_cast<int>(min(64u, rows - r0));
    if (tid < 64) {
      float* x = xin + tid * kSurrIn;
      if (tid < nvalid) {
        event_row(qne[r0 + tid], nuc_slot, key, x);
      } else {
        for (int j = 0; j < kSurrIn; ++j) x[j] = 0.0f;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      for (int e = tid; e < 64 * kSurrIn; e += 128) {
        const int r = e / kSurrIn, c = e % kSurrIn;
        tile[r * kActLd + c] = __float2bfloat16_rn(xin[r * kSurrIn + c]);
      }
      mlp_tile(tile, Wb, P, pass == 0 ? y1 : y2, nvalid);
      __syncthreads();
      if (pass == 0 && tid < nvalid)
        xin[tid * kSurrIn + 1 + kSurrTargets] = static_cast<float>(multiplicity(y1[tid * kSurrOut])) / kSurrSlots;
      __syncthreads();
    }
    if (tid < nvalid)
      emit_event(qne[r0 + tid], y1 + tid * kSurrOut, y2 + tid * kSurrOut, key, tally, B, qsec, qsec_count, qsec_cap,
                 hist, hist_n, dep, esc, sec, dropped);
    __syncthreads();
  }
  auto wsum = [](unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  const unsigned long long d = wsum(static_cast<unsigned long long>(dep)), e = wsum(static_cast<unsigned long long>(esc));
  const unsigned long long s = wsum(sec), dr = wsum(dropped);
  if ((threadIdx.x & 31) == 0) {
    if (d) atomicAdd(&cnt->deposited, d);
    if (e) atomicAdd(&cnt->escaped, e);
    if (s) atomicAdd(&cnt->secondaries, s);
    if (dr) atomicAdd(&cnt->dropped, dr);
  }
}

__global__ void to_bf16_kernel(int n, const float* a, __nv_bfloat16* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

cudaError_t launch_mlp_infer(const unsigned* n_rows, unsigned cap, const float* X, const void* Wb, const float* P,
                             float* Y, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  mlp_infer_kernel<<<grid, 128, kInferSmem, s>>>(n_rows, cap, X, static_cast<const __nv_bfloat16*>(Wb), P, Y);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(int n, const float* a, void* b, cudaStream_t s) {
  to_bf16_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, static_cast<__nv_bfloat16*>(b));
  return cudaGetLastError();
}

cudaError_t launch_gemm(int M, const unsigned* Mp, int N, int K, const float* A, long long sam, long long sak,
                        const float* B, long long sbk, long long sbn, float* C, long long ldc, const float* bias,
                        bool relu, const float* mask, bool accumulate, cudaStream_t s) {
  const dim3 grid((M + kTileM - 1) / kTileM, (N + kTileN - 1) / kTileN);
  gemm_kernel<<<grid, 128, 0, s>>>(M, Mp, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu ? 1 : 0, mask,
                                   accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_pinball(int rows, const float* yhat, const float* y, const float* tau, const float* mask,
                           float* grad, float* loss, cudaStream_t s) {
  const int n = rows * kSurrOut;
  pinball_kernel<<<(n + 255) / 256, 256, 0, s>>>(rows, yhat, y, tau, mask, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_colsum(int rows, int N, const float* G, float* db, cudaStream_t s) {
  colsum_kernel<<<N, 256, 0, s>>>(rows, N, G, db);
  return cudaGetLastError();
}

cudaError_t launch_adamw(int n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                         float wd, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, static_cast<float>(step)), c2 = 1.0f - powf(b2, static_cast<float>(step));
  adamw_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, p, g, m, v, lr, b1, b2, eps, wd, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_train_rows(int batch, const float* feat, const unsigned* perm, unsigned long long first,
                              unsigned long long n_events, unsigned long long seed, unsigned step, float* X, float* Y,
                              float* tau, float* mask, cudaStream_t s) {
  train_rows_kernel<<<(2 * batch + 127) / 128, 128, 0, s>>>(batch, feat, perm, first, n_events, seed, step, X, Y, tau,
                                                             mask);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_events(const unsigned* n_ev, unsigned cap, const Particle* qne, const int* nuc_slot,
                                    const unsigned long long* seed, const void* Wb, const float* P,
                                    unsigned long long* tally, int B, Particle* qsec, unsigned* qsec_count,
                                    unsigned qsec_cap, Counters* cnt, long long* hist, unsigned long long hist_n,
                                    int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(surrogate_event_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kEventSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  surrogate_event_kernel<<<grid, 128, kEventSmem, s>>>(n_ev, cap, qne, nuc_slot, seed,
                                                        static_cast<const __nv_bfloat16*>(Wb), P, tally, B, qsec,
                                                        qsec_count, qsec_cap, cnt, hist, hist_n);
  return cudaGetLastError();
}

}  // namespace pmc
