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
// Dense layers run on the 5th-generation tensor cores (tcgen05 MMAs, BF16 operands,
// FP32 accumulators in tensor memory; namespace tc below): inference (the event stage
// inside the transport, and pmc_surrogate_infer) and the training GEMMs (forward and both
// backward products, from FP32 master copies rounded when a tile is staged in shared
// memory).
#include <cuda_bf16.h>

#include "pmc_kernels.cuh"

namespace pmc {
namespace {

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
// (x is the thread's own row, kept in registers: every index below is a compile-time one)
__device__ __forceinline__ void event_row(const Particle& ev, const int* nuc_slot, uint2 key, float (&x)[kSurrIn]) {
#pragma unroll
  for (int j = 0; j < kSurrIn; ++j) x[j] = 0.0f;
  x[0] = (ev.E - 130.0f) / 120.0f;
  const int slot = nuc_slot[ev.target];
#pragma unroll
  for (int j = 0; j < kSurrTargets; ++j) x[1 + j] = j == slot ? 1.0f : 0.0f;
  x[1 + kSurrTargets] = -1.0f;
  const float4 u0 = draw4(key, ev.pid, 0u, 8u), u1 = draw4(key, ev.pid, 1u, 8u), u2 = draw4(key, ev.pid, 2u, 8u);
  const float u[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
#pragma unroll
  for (int j = 0; j < kSurrTau; ++j) x[2 + kSurrTargets + j] = u[j];
}

__device__ __forceinline__ int multiplicity(float q) {
  return min(max(static_cast<int>(floorf(q + 0.5f)), 0), kSurrSlots);
}

// Emits an event from the network's quantiles: protons to the secondary queue,
// the local deposit to the event voxel, the rest (neutrons, photons, binding)
// escapes.  Energy is conserved by construction.
__device__ void emit_event(const Particle& ev, const float (&y1)[kSurrOut], const float (&y2)[kSurrOut], uint2 key,
                           unsigned long long* tally,
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
  // the protons above the cut take queue slots by one atomic per group of converged lanes:
  // slot k of every lane, in lane order, then slot k + 1 (the queue's order is immaterial:
  // each proton's random numbers follow from its identity)
  static_assert(kSurrSlots <= 4, "four azimuth uniforms per event");
  const unsigned mask = __activemask(), lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
  const int leader = __ffs(mask) - 1;
  unsigned bk[kSurrSlots], total = 0;
#pragma unroll
  for (int k = 0; k < kSurrSlots; ++k) {
    bk[k] = __ballot_sync(mask, k < np && T[k] > kEcut);
    total += __popc(bk[k]);
  }
  unsigned base = 0;
  if (static_cast<int>(lane) == leader && total) base = atomicAdd(qsec_count, total);
  base = __shfl_sync(mask, base, leader);
  long long handed = 0;
#pragma unroll
  for (int k = 0; k < kSurrSlots; ++k) {
    const unsigned off = base + __popc(bk[k] & lt);
    base += __popc(bk[k]);
    if (k >= np) continue;
    if (T[k] <= kEcut) { loc += T[k]; continue; }
    float sp, cp;
    sincospif(2.0f * uphi[k], &sp, &cp);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - c[k] * c[k]));
    const float3 d = frame_to_lab(ev.u, ev.v, ev.w, st * cp, st * sp, c[k]);
    Particle r;
    r.x = ev.x; r.y = ev.y; r.z = ev.z; r.u = d.x; r.v = d.y; r.w = d.z; r.E = T[k];
    r.voxel = ev.voxel; r.pid = child_pid(key, ev.pid, static_cast<unsigned>(k)); r.root = ev.root; r.target = -1;
    if (off < qsec_cap) {
      qsec[off] = r;
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

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): the network of the event stage on 128-row tiles.
// Operands live in shared memory in the canonical K-major layout without swizzle: "core
// matrices" of 8 rows x 16 bytes (8 BF16 along K), contiguous (128 B); the two core matrices
// of a 16-wide K slice sit 128 B apart (leading byte offset) and successive 8-row groups
// 256 B apart (stride byte offset), so one K slice of 128 rows is 4 KB.  One thread issues
// the MMAs (D[128 x N] += A[128 x 16] B[16 x N], BF16 in, FP32 accumulate in tensor memory);
// their completion is signalled on an mbarrier, and the epilogue reads the accumulator back
// with tcgen05.ld (warp w owns accumulator rows 32w..32w+31).
// ---------------------------------------------------------------------------
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, bool accumulate) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(a), "l"(b), "r"(id), "r"(accumulate ? 1 : 0));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Waits for the mbarrier phase with the given parity; false after `spin` polls (the caller
// reports the error and stops issuing work).
constexpr int kSpin = 1 << 22;
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity, int spin) {
  uint32_t done = 0;
  for (int it = 0; it < spin && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
  return done != 0;
}

// 16 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

static_assert(kSurrHidden % 64 == 0, "the epilogue reads the hidden layers 64 columns at a time");
// 64 consecutive FP32 accumulator columns of this thread's row, one load and one wait.
__device__ __forceinline__ void ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offsets in the canonical layout: activation (row r, column k) of the 128-row tile, and
// weight (output n, chunk column kl) of a chunk of kKC columns for N outputs.
constexpr int kRows = 128, kKC = 32;
__device__ __forceinline__ uint32_t act_off(int r, int k) {
  return (k >> 4) * 4096 + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t w_off(int n, int kl, int N) {
  return (kl >> 4) * (N * 32) + (n >> 3) * 256 + ((kl >> 3) & 1) * 128 + (n & 7) * 16 + (kl & 7) * 2;
}

constexpr int kActBytes = 16 * 4096;                 // 128 rows x 256 BF16
constexpr int kWBytes = kSurrHidden * kKC * 2;       // one weight chunk: 256 outputs x 32 columns
constexpr int kStages = 3;                           // weight-chunk buffers (two chunks in flight)
constexpr int kTmemCols = kSurrHidden;               // the widest accumulator: 128 x 256 FP32

__device__ __forceinline__ int layer_in(int l) { return l == 0 ? kSurrIn : kSurrHidden; }
__device__ __forceinline__ int layer_out(int l) { return l == kSurrLayers - 1 ? kSurrOut : kSurrHidden; }

// The packed weights: every chunk of a layer (a run of its input columns) stored contiguously in
// exactly the byte order of its shared-memory buffer (w_off), so that one bulk copy moves it.
// A chunk is as many 16-wide K slices as fill one buffer, at most the layer's whole K: kKC
// columns of the 256-wide layers, all 256 of the 16-wide output layer (8 KB, one copy rather
// than eight round trips).  A pass streams kChunksPerPass chunks.
__host__ __device__ constexpr int layer_in_c(int l) { return l == 0 ? kSurrIn : kSurrHidden; }
__host__ __device__ constexpr int layer_out_c(int l) { return l == kSurrLayers - 1 ? kSurrOut : kSurrHidden; }
__host__ __device__ constexpr int chunk_cols(int l) {
  return kWBytes / (2 * layer_out_c(l)) < layer_in_c(l) ? kWBytes / (2 * layer_out_c(l)) : layer_in_c(l);
}
__host__ __device__ constexpr int layer_chunks(int l) { return layer_in_c(l) / chunk_cols(l); }
__host__ __device__ constexpr int chunks_per_pass() {
  int n = 0;
  for (int l = 0; l < kSurrLayers; ++l) n += layer_chunks(l);
  return n;
}
constexpr int kChunksPerPass = chunks_per_pass();
static_assert(chunk_cols(0) % 16 == 0 && chunk_cols(kSurrLayers - 1) % 16 == 0 && kKC % 16 == 0,
              "chunks are whole 16-wide K slices");
// Chunk k of the pass -> its layer and column chunk.
__device__ __forceinline__ void chunk_pos(int k, int& l, int& c) {
  l = 0;
  while (k >= layer_chunks(l)) {
    k -= layer_chunks(l);
    ++l;
  }
  c = k;
}
// Byte offset of chunk (l, c) in the packed weights, and its size.
__host__ __device__ inline size_t chunk_offset(int l, int c) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += static_cast<size_t>(layer_in_c(i)) * layer_out_c(i) * 2;
  return o + static_cast<size_t>(c) * layer_out_c(l) * chunk_cols(l) * 2;
}
__host__ __device__ constexpr uint32_t chunk_bytes(int l) { return static_cast<uint32_t>(layer_out_c(l) * chunk_cols(l) * 2); }

// Pipeline state kept across passes.  Barriers at mbar + 8 i: full[b] (i = b: the bulk copy
// of the chunk in buffer b has landed), empty[b] (i = kStages + b: the MMAs reading buffer b
// are done), layer (i = 2 kStages: all MMAs of a layer are done).  Thread 0 runs the chunk
// stream and waits on full and empty; every thread waits on layer.  Each completion of each
// barrier is waited exactly once, so a parity bit per barrier tracks its phase.
struct Pipe {
  uint32_t tmem, mbar, phase;   // phase bit i: parity of barrier i's next completion
  bool ok;
  bool issue;                   // false only in the wait check: no MMA is issued, so waits run out
  int spin;                     // polls per wait
  int issued;                   // thread 0: chunks of the current pass whose copies were started
  bool pre;                     // thread 0: the next pass's first kStages copies are already started
  __device__ __forceinline__ uint32_t bar(int i) const { return mbar + 8u * i; }
  // A copy always lands, so the "full" waits keep the long bound even in the wait check: only
  // the waits on MMAs run out there, and no copy is left in flight when the block stops.
  __device__ __forceinline__ bool wait_bar(int i) {
    const bool r = wait(bar(i), (phase >> i) & 1u, i < kStages ? kSpin : spin);
    phase ^= 1u << i;
    return r;
  }
};

// Thread 0: starts the bulk copy of chunk k of the pass into its buffer.  Chunk k goes to
// buffer k % kStages (the pass's stream position, whatever the chunk's size).
__device__ __forceinline__ void issue_copy(Pipe& pp, int k, const unsigned char* __restrict__ packed,
                                           unsigned char* wb) {
  int l, c;
  chunk_pos(k, l, c);
  const int b = k % kStages;
  const uint32_t bytes = chunk_bytes(l);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pp.bar(b)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(saddr(wb + b * kWBytes)), "l"(packed + chunk_offset(l, c)), "r"(bytes), "r"(pp.bar(b))
               : "memory");
  pp.issued = k + 1;
}

// Thread 0, chunk q's MMAs issued (or, with q one past a layer's last chunk, that layer's MMAs
// all done): refills the buffer of chunk q-1 with chunk q-1+kStages once chunk q-1's MMAs are
// done, unless that copy was already started.  Every chunk's "empty" completion is waited
// exactly once: here, or at the end of the pass for the last kStages chunks.
__device__ __forceinline__ void refill(Pipe& pp, int q, const unsigned char* __restrict__ packed, unsigned char* wb) {
  if (pp.ok && q >= 1 && pp.issued == q - 1 + kStages && pp.issued < kChunksPerPass) {
    pp.ok = pp.wait_bar(kStages + (q - 1) % kStages);
    if (pp.ok) issue_copy(pp, q - 1 + kStages, packed, wb);
  }
}

// One pass of the network over the tile: inputs in act columns 0..kSurrIn-1 (written by every
// thread before the call); each thread's row of the last layer (bias added) goes to its
// registers out[n].  Thread 0 streams the weight chunks by bulk copies kStages deep and issues
// the MMAs; after issuing chunk q's it refills the buffer of chunk q-1 (whose MMAs have had
// chunk q's time to finish), and at a layer's end the buffer of its last chunk as soon as the
// layer's MMAs are done, so that the next layer's chunks load during the epilogue.  All threads
// meet at each layer's end for the epilogue.  With `next` (another pass follows on this block),
// thread 0 starts that pass's first copies as soon as this pass's MMAs are done.
__device__ __forceinline__ void mlp_pass(unsigned char* act, unsigned char* wb, Pipe& pp,
                                         const unsigned char* __restrict__ packed, const float* __restrict__ P,
                                         float (&out)[kSurrOut], bool next) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t trow = pp.tmem + (static_cast<uint32_t>(warp * 32) << 16);
  if (tid == 0) {
    if (!pp.pre) {
      pp.issued = 0;
      if (pp.ok)
        for (int k = 0; k < kStages; ++k) issue_copy(pp, k, packed, wb);
    }
    pp.pre = false;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the layer-0 operand rows
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  size_t off = 0;
  int q = 0;
#pragma unroll 1
  for (int l = 0; l < kSurrLayers; ++l) {
    const int din = layer_in_c(l), N = layer_out_c(l), cs = chunk_cols(l) / 16, nc = din / chunk_cols(l);
    const float* __restrict__ bias = P + off + static_cast<size_t>(din) * N;
    if (tid == 0) {
      const uint32_t id = idesc(kRows, N);
#pragma unroll 1
      for (int c = 0; c < nc; ++c, ++q) {
        const int b = q % kStages;
        if (q < pp.issued) pp.ok = pp.wait_bar(b) && pp.ok;   // the chunk landed (waited even after a failure)
        if (pp.ok && pp.issue) {
#pragma unroll 1
          for (int s2 = 0; s2 < cs; ++s2)
            mma(pp.tmem, desc(saddr(act + (c * cs + s2) * 4096), 128, 256),
                desc(saddr(wb + b * kWBytes + s2 * (N * 32)), 128, 256), id, c > 0 || s2 > 0);
          commit(pp.bar(kStages + b));
          if (c + 1 == nc) commit(pp.bar(2 * kStages));
        }
        refill(pp, q, packed, wb);
      }
    }
    // every thread: the layer's MMAs are done (warp-uniform outcome: tcgen05.ld is warp-collective)
    const bool r = pp.ok && wait(pp.bar(2 * kStages), (pp.phase >> (2 * kStages)) & 1u, pp.spin);
    pp.phase ^= 1u << (2 * kStages);
    pp.ok = __all_sync(0xffffffffu, r);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) refill(pp, q, packed, wb);   // the layer's last buffer: free now
    pp.ok = __all_sync(0xffffffffu, pp.ok);     // warp 0 stays converged and of one mind for tcgen05.ld
    if (pp.ok) {
      if (l + 1 < kSurrLayers) {
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 64) {   // 64 columns per tensor-memory load (one wait)
          float v[64];
          ld64(trow + c0, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            // the bias of a hidden layer starts on a 64-byte boundary of P (every block of P is a
            // multiple of 16 floats long), so eight columns are two 16-byte loads
            const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * q));
            const float4 b1 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * q + 4));
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            uint32_t h[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int c = 8 * q + 2 * i;
              const __nv_bfloat162 t2 = __floats2bfloat162_rn(fmaxf(v[c] + bb[2 * i], 0.0f),
                                                              fmaxf(v[c + 1] + bb[2 * i + 1], 0.0f));
              h[i] = *reinterpret_cast<const uint32_t*>(&t2);
            }
            *reinterpret_cast<uint4*>(act + act_off(tid, c0 + 8 * q)) = make_uint4(h[0], h[1], h[2], h[3]);
          }
        }
      } else {
        float v[16];
        ld16(trow, v);
#pragma unroll
        for (int i = 0; i < kSurrOut; ++i) out[i] = v[i] + __ldg(bias + i);
      }
    }
    off += static_cast<size_t>(din) * N + N;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the epilogue's operand rows
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // thread 0: the MMA completions of the last chunks, whose buffers were not refilled; then,
  // with another pass to come, that pass's first copies into the freed buffers
  if (tid == 0 && pp.ok && pp.issue) {
    for (int k = kChunksPerPass - kStages; k < kChunksPerPass; ++k) pp.ok = pp.wait_bar(kStages + k % kStages) && pp.ok;
    if (pp.ok && next) {
      pp.issued = 0;
      for (int k = 0; k < kStages; ++k) issue_copy(pp, k, packed, wb);
      pp.pre = true;
    }
  }
}
static_assert(kChunksPerPass > kStages, "the stream is deeper than the pipeline");

// Setup of a block that runs the network on the tensor cores (every thread calls it): 2 kStages
// + 1 mbarriers and kTmemCols columns of tensor memory, allocated by warp 0.
__device__ __forceinline__ Pipe begin(unsigned long long* mbar, uint32_t* tslot, int* fail, bool issue = true,
                                      int spin = kSpin) {
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 * kStages + 1; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar + b)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail = 0;
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return Pipe{*tslot, saddr(mbar), 0u, true, issue, spin, 0, false};
}

// Frees the block's tensor memory (every thread calls it, after its last tcgen05.ld), with no
// copy of its own still in flight: thread 0 first waits (bounded) for the copies it started for
// a pass that did not run (a block that stopped on a failure).
__device__ __forceinline__ void end(Pipe& pp) {
  if (threadIdx.x == 0 && pp.pre)
    for (int k = 0; k < kStages; ++k) pp.wait_bar(k);
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(pp.tmem), "r"(kTmemCols));
}

// This thread's row of the layer-0 operand from FP32 inputs (BF16, canonical layout).
__device__ __forceinline__ void put_row(unsigned char* act, const float (&x)[kSurrIn]) {
#pragma unroll
  for (int k0 = 0; k0 < kSurrIn; k0 += 8) {
    uint32_t h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 t2 = __floats2bfloat162_rn(x[k0 + 2 * i], x[k0 + 2 * i + 1]);
      h[i] = *reinterpret_cast<const uint32_t*>(&t2);
    }
    *reinterpret_cast<uint4*>(act + act_off(threadIdx.x, k0)) = make_uint4(h[0], h[1], h[2], h[3]);
  }
}

// Shared memory of a network block (the descriptors need 16-byte alignment, which dynamic
// shared memory has; bulk copies 16-byte addresses and sizes): activations, the weight buffers,
// 2 kStages + 1 mbarriers, the tensor-memory address and a failure flag.  112 KB: two blocks
// per SM, each with 256 TMEM columns.
struct Smem {
  unsigned char *act, *wb;
  unsigned long long* mbar;
  uint32_t* tslot;
  int* fail;
};
__device__ __forceinline__ Smem carve(unsigned char* smem) {
  Smem m;
  m.act = smem;
  m.wb = m.act + kActBytes;
  m.mbar = reinterpret_cast<unsigned long long*>(m.wb + kStages * kWBytes);
  m.tslot = reinterpret_cast<uint32_t*>(m.mbar + 2 * kStages + 1);
  m.fail = reinterpret_cast<int*>(m.tslot + 1);
  return m;
}
constexpr int kSmem = kActBytes + kStages * kWBytes + 8 * (2 * kStages + 1) + 8;

}  // namespace tc

// The network over rows X[n][kSurrIn] -> Y[n][kSurrOut] (persistent over 128-row tiles); a
// tensor-core wait that timed out raises *err.  With check_waits the MMAs are withheld and the
// waits poll briefly: they run out, which exercises the error path (nothing is in flight).
__global__ void __launch_bounds__(128, 2) mlp_rows_kernel(int rows, const float* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ Wb,
                                                         const float* __restrict__ P, float* __restrict__ Y, int* err,
                                                         int check_waits) {
  extern __shared__ __align__(16) unsigned char smem[];
  const tc::Smem m = tc::carve(smem);
  const int tid = threadIdx.x;
  if (rows <= static_cast<int>(blockIdx.x) * tc::kRows) return;   // uniform: no tensor memory taken
  tc::Pipe pp = tc::begin(m.mbar, m.tslot, m.fail, !check_waits, check_waits ? 256 : tc::kSpin);
  for (int r0 = blockIdx.x * tc::kRows; r0 < rows; r0 += gridDim.x * tc::kRows) {
    const int nvalid = min(tc::kRows, rows - r0);
    float x[kSurrIn], y[kSurrOut];
#pragma unroll
    for (int j = 0; j < kSurrIn; ++j) x[j] = tid < nvalid ? X[static_cast<size_t>(r0 + tid) * kSurrIn + j] : 0.0f;
    tc::put_row(m.act, x);
    tc::mlp_pass(m.act, m.wb, pp, reinterpret_cast<const unsigned char*>(Wb), P, y,
                 r0 + gridDim.x * tc::kRows < rows);
    if (!pp.ok) atomicOr(m.fail, 1);
    __syncthreads();
    if (*m.fail) break;
    if (tid < nvalid) {
#pragma unroll
      for (int j = 0; j < kSurrOut; ++j) Y[static_cast<size_t>(r0 + tid) * kSurrOut + j] = y[j];
    }
  }
  if (tid == 0 && *m.fail) atomicAdd(err, 1);
  tc::end(pp);
}

// The event stage of the primaries' events with the learned stand-in, fused: per tile of 128 queued
// events (one per thread), build the inference rows, run the network on the tensor cores
// (multiplicity pass), condition on the sampled multiplicity, run it again and emit the
// events, with rows, activations and outputs in shared memory throughout.
__global__ void __launch_bounds__(128, 2) surrogate_event_kernel(const unsigned* n_ev, unsigned cap,
                                                              const Particle* __restrict__ qne, const int* nuc_slot,
                                                              const unsigned long long* seedp,
                                                              const __nv_bfloat16* __restrict__ Wb,
                                                              const float* __restrict__ P, unsigned long long* tally,
                                                              int B, Particle* qsec, unsigned* qsec_count,
                                                              unsigned qsec_cap, Counters* cnt, long long* hist,
                                                              unsigned long long hist_n) {
  extern __shared__ __align__(16) unsigned char smem[];
  const tc::Smem m = tc::carve(smem);
  const int tid = threadIdx.x;
  const unsigned rows = min(*n_ev, cap);
  if (rows <= static_cast<unsigned>(blockIdx.x) * tc::kRows) return;   // uniform: no tensor memory taken
  tc::Pipe pp = tc::begin(m.mbar, m.tslot, m.fail);
  const unsigned long long seed = *seedp;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  long long dep = 0, esc = 0;
  unsigned long long sec = 0, dropped = 0, n_done = 0;
  for (unsigned r0 = blockIdx.x * tc::kRows; r0 < rows; r0 += gridDim.x * tc::kRows) {
    const int nvalid = static_cast<int>(min(static_cast<unsigned>(tc::kRows), rows - r0));
    float x[kSurrIn], y1[kSurrOut], y2[kSurrOut];
    if (tid < nvalid) {
      event_row(qne[r0 + tid], nuc_slot, key, x);
    } else {
#pragma unroll
      for (int j = 0; j < kSurrIn; ++j) x[j] = 0.0f;
    }
    tc::put_row(m.act, x);
    tc::mlp_pass(m.act, m.wb, pp, reinterpret_cast<const unsigned char*>(Wb), P, y1, true);   // multiplicity pass
    x[1 + kSurrTargets] = static_cast<float>(multiplicity(y1[0])) / kSurrSlots;
    tc::put_row(m.act, x);
    tc::mlp_pass(m.act, m.wb, pp, reinterpret_cast<const unsigned char*>(Wb), P, y2,
                 r0 + gridDim.x * tc::kRows < rows);                                         // conditioned on it
    if (!pp.ok) atomicOr(m.fail, 1);
    __syncthreads();
    if (*m.fail) break;                               // a tensor-core wait timed out: stop
    if (tid < nvalid)
      emit_event(qne[r0 + tid], y1, y2, key, tally, B, qsec, qsec_count, qsec_cap, hist, hist_n, dep, esc, sec,
                 dropped);
    n_done += static_cast<unsigned long long>(nvalid);
  }
  auto wsum = [](unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  const unsigned long long d = wsum(static_cast<unsigned long long>(dep)), e = wsum(static_cast<unsigned long long>(esc));
  const unsigned long long s2 = wsum(sec), dr = wsum(dropped);
  if ((tid & 31) == 0) {
    if (d) atomicAdd(&cnt->deposited, d);
    if (e) atomicAdd(&cnt->escaped, e);
    if (s2) atomicAdd(&cnt->secondaries, s2);
    if (dr) atomicAdd(&cnt->dropped, dr);
  }
  if (tid == 0 && *m.fail) atomicAdd(&cnt->errors, 1ull);
  if (tid == 0 && n_done) atomicAdd(&cnt->surrogate_events, n_done);
  tc::end(pp);
}

// ---------------------------------------------------------------------------
// Training GEMM on the 5th-generation tensor cores.  C[m][n] (=|+=) sum_k A(m,k) B(k,n)
// (+ bias[n]) (ReLU) (* [mask[m][n] > 0]), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn],
// FP32 in memory, BF16 operands, FP32 accumulation in tensor memory.  One CTA (4 warps) owns a
// 128 x BN tile (BN <= 256) and a range of K: each 64-wide K chunk is loaded by all threads
// (FP32 -> BF16, written into the canonical no-swizzle K-major layout of the inference kernel,
// transposed on the way when the source is M- or N-major), then one thread issues its
// tcgen05 MMAs and commits them to the chunk's buffer mbarrier; two buffers, so the next
// chunk loads while the MMAs run.  With a K split (the weight gradients, whose K is the batch),
// each CTA writes its partial tile to a workspace that gemm_reduce_kernel sums in a fixed
// order (deterministic) before the epilogue.
// ---------------------------------------------------------------------------
constexpr int kGemmBK = 64;
constexpr int kGemmABytes = tc::kRows * kGemmBK * 2;            // 16 KB
constexpr int kGemmBBytes = 256 * kGemmBK * 2;                  // 32 KB at BN = 256
constexpr int kGemmSmem = 2 * (kGemmABytes + kGemmBBytes) + 64;

__device__ __forceinline__ void gemm_epilogue(float v, int m, int n, float* C, long long ldc, const float* bias,
                                              int relu, const float* mask, int accumulate) {
  if (bias) v += bias[n];
  if (relu) v = fmaxf(v, 0.0f);
  if (mask && !(mask[static_cast<long long>(m) * ldc + n] > 0.0f)) v = 0.0f;
  float* dst = C + static_cast<long long>(m) * ldc + n;
  *dst = accumulate ? *dst + v : v;
}

// Eight consecutive k of one row (of A) or one column (of B) as a 16-byte BF16 unit.
__device__ __forceinline__ uint4 load_unit(const float* __restrict__ X, long long s_row, long long s_k, int row,
                                           int rows, int k, int kend) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    v[j] = (row < rows && k + j < kend) ? X[static_cast<long long>(row) * s_row + static_cast<long long>(k + j) * s_k]
                                        : 0.0f;
  uint32_t h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 t2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    h[i] = *reinterpret_cast<const uint32_t*>(&t2);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, int BN, int k_split,
                                                      const float* __restrict__ A, long long sam, long long sak,
                                                      const float* __restrict__ B, long long sbk, long long sbn,
                                                      float* __restrict__ C, long long ldc,
                                                      const float* __restrict__ bias, int relu,
                                                      const float* __restrict__ mask, int accumulate,
                                                      float* __restrict__ ws, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* abuf[2] = {smem, smem + kGemmABytes};
  unsigned char* bbuf[2] = {smem + 2 * kGemmABytes, smem + 2 * kGemmABytes + kGemmBBytes};
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + 2 * (kGemmABytes + kGemmBBytes));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
  int* fail = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * tc::kRows, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * k_split, kend = min(K, kbeg + k_split);
  const int ncols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));   // tensor-memory columns
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(mbar + b)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(tslot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const bool a_mfast = sam == 1, b_nfast = sbn == 1;   // the operand's contiguous direction
  const uint32_t id = tc::idesc(tc::kRows, BN);
  const int nchunks = (kend - kbeg + kGemmBK - 1) / kGemmBK;
  uint32_t phase = 0;   // bit b: parity of buffer b's next completion; bit 2: the final barrier
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1, k0 = kbeg + c * kGemmBK;
    if (c >= 2) {   // the MMAs that read this buffer two chunks ago are done
      ok = tc::wait(tc::saddr(mbar + b), (phase >> b) & 1u, tc::kSpin) && ok;
      phase ^= 1u << b;
    }
    // A: 128 rows x 64 k (1024 units of 8 k), B: BN columns x 64 k
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
      const int u = tid + 128 * i;
      const int r = a_mfast ? (u & 127) : (u >> 3), k8 = a_mfast ? (u >> 7) : (u & 7);
      *reinterpret_cast<uint4*>(abuf[b] + tc::act_off(r, 8 * k8)) = load_unit(A, sam, sak, m0 + r, M, k0 + 8 * k8, kend);
    }
    for (int u = tid; u < BN * 8; u += 128) {
      const int nn = b_nfast ? (u % BN) : (u >> 3), k8 = b_nfast ? (u / BN) : (u & 7);
      *reinterpret_cast<uint4*>(bbuf[b] + tc::w_off(nn, 8 * k8, BN)) =
          load_unit(B, sbn, sbk, n0 + nn, N, k0 + 8 * k8, kend);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && ok) {
      const int nks = (min(kGemmBK, kend - k0) + 15) / 16;
      for (int s = 0; s < nks; ++s)
        tc::mma(tmem, tc::desc(tc::saddr(abuf[b] + s * 4096), 128, 256), tc::desc(tc::saddr(bbuf[b] + s * (BN * 32)), 128, 256),
                id, c > 0 || s > 0);
      tc::commit(tc::saddr(mbar + b));
      if (c + 1 == nchunks) tc::commit(tc::saddr(mbar + 2));
    }
  }
  // every MMA of the tile is done (the last commit tracks all earlier ones)
  if (nchunks > 0) ok = tc::wait(tc::saddr(mbar + 2), (phase >> 2) & 1u, tc::kSpin) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __all_sync(0xffffffffu, ok);   // warp-uniform: tcgen05.ld is warp-collective
  if (!ok) atomicOr(fail, 1);
  if (ok) {
    const int m = m0 + warp * 32 + (tid & 31);
    const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc::ld16(trow + c0, v);
      if (m >= M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = n0 + c0 + i;
        if (n >= N) break;
        if (ws) ws[(static_cast<long long>(blockIdx.z) * M + m) * N + n] = v[i];
        else gemm_epilogue(v[i], m, n, C, ldc, bias, relu, mask, accumulate);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  if (tid == 0 && *fail) atomicAdd(err, 1);
}

// The K split's partial tiles summed in split order, then the epilogue.
__global__ void gemm_reduce_kernel(int M, int N, int splits, const float* __restrict__ ws, float* __restrict__ C,
                                   long long ldc, const float* __restrict__ bias, int relu,
                                   const float* __restrict__ mask, int accumulate) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(M) * N) return;
  const int m = static_cast<int>(i / N), n = static_cast<int>(i % N);
  float v = 0.0f;
  for (int z = 0; z < splits; ++z) v += ws[(static_cast<long long>(z) * M + m) * N + n];
  gemm_epilogue(v, m, n, C, ldc, bias, relu, mask, accumulate);
}

// The inference weights: BF16 of the FP32 parameters (round to nearest even), each chunk in
// the byte order of its shared-memory buffer (one 16-byte unit = 8 consecutive columns of one
// output row per thread).
__global__ void pack_weights_kernel(const float* __restrict__ P, unsigned char* __restrict__ packed) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  size_t off = 0;
  for (int l = 0; l < kSurrLayers; ++l) {
    const int din = tc::layer_in_c(l), N = tc::layer_out_c(l), units = N * din / 8;
    if (u < units) {
      const int n = u / (din / 8), k = (u % (din / 8)) * 8, c = k / tc::chunk_cols(l), kl = k % tc::chunk_cols(l);
      const float* w = P + off + static_cast<size_t>(n) * din + k;
      uint32_t h[4];
      for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 t2 = __floats2bfloat162_rn(w[2 * i], w[2 * i + 1]);
        h[i] = *reinterpret_cast<const uint32_t*>(&t2);
      }
      *reinterpret_cast<uint4*>(packed + tc::chunk_offset(l, c) + tc::w_off(n, kl, N)) = make_uint4(h[0], h[1], h[2], h[3]);
      return;
    }
    u -= units;
    off += static_cast<size_t>(din) * N + N;
  }
}

}  // namespace

cudaError_t launch_mlp_rows(int rows, const float* X, const void* Wb, const float* P, float* Y, int* err, int n_sm,
                            bool check_waits, cudaStream_t s) {
  // set once per process; a function-local static is initialised exactly once even when
  // several host threads (the multi-plan stream's slots) reach this first
  static const cudaError_t attr = cudaFuncSetAttribute(mlp_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem);
  if (attr != cudaSuccess) return attr;
  const int grid = min(2 * n_sm, (rows + tc::kRows - 1) / tc::kRows);
  mlp_rows_kernel<<<grid, tc::kRows, tc::kSmem, s>>>(rows, X, static_cast<const __nv_bfloat16*>(Wb), P, Y, err,
                                                     check_waits ? 1 : 0);
  return cudaGetLastError();
}

size_t packed_weight_bytes() { return tc::chunk_offset(kSurrLayers, 0); }

cudaError_t launch_pack_weights(const float* P, void* packed, cudaStream_t s) {
  const int units = static_cast<int>(packed_weight_bytes() / 16);
  pack_weights_kernel<<<(units + 255) / 256, 256, 0, s>>>(P, static_cast<unsigned char*>(packed));
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(int M, int N, int K, const float* A, long long sam, long long sak, const float* B,
                          long long sbk, long long sbn, float* C, long long ldc, const float* bias, bool relu,
                          const float* mask, bool accumulate, float* ws, size_t ws_floats, int* err, int n_sm,
                          cudaStream_t s) {
  // set once per process (a function-local static is initialised exactly once)
  static const cudaError_t attr = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  if (attr != cudaSuccess) return attr;
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  const int BN = min(256, (N + 15) / 16 * 16);
  const int mt = (M + tc::kRows - 1) / tc::kRows, nt = (N + BN - 1) / BN;
  const int kchunks = (K + kGemmBK - 1) / kGemmBK;
  // split K when the tiles alone would leave most SMs idle (the weight gradients: K = batch rows)
  int splits = 1;
  if (ws && 2 * mt * nt < n_sm) {
    splits = min(kchunks, (2 * n_sm + mt * nt - 1) / (mt * nt));
    while (splits > 1 && static_cast<size_t>(splits) * M * N > ws_floats) --splits;
  }
  const int k_split = (kchunks + splits - 1) / splits * kGemmBK;
  splits = (K + k_split - 1) / k_split;   // every split has at least one chunk
  const dim3 grid(mt, nt, splits);
  gemm_tc_kernel<<<grid, tc::kRows, kGemmSmem, s>>>(M, N, K, BN, k_split, A, sam, sak, B, sbk, sbn, C, ldc, bias,
                                                    relu ? 1 : 0, mask, accumulate ? 1 : 0, splits > 1 ? ws : nullptr,
                                                    err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const long long total = static_cast<long long>(M) * N;
  gemm_reduce_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(M, N, splits, ws, C, ldc, bias,
                                                                                relu ? 1 : 0, mask, accumulate ? 1 : 0);
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
  // set once per process; a function-local static is initialised exactly once even when
  // several host threads (the multi-plan stream's slots) reach this first
  static const cudaError_t attr = cudaFuncSetAttribute(surrogate_event_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem);
  if (attr != cudaSuccess) return attr;
  surrogate_event_kernel<<<grid, tc::kRows, tc::kSmem, s>>>(n_ev, cap, qne, nuc_slot, seed,
                                                        static_cast<const __nv_bfloat16*>(Wb), P, tally, B, qsec,
                                                        qsec_count, qsec_cap, cnt, hist, hist_n);
  return cudaGetLastError();
}

}  // namespace pmc
