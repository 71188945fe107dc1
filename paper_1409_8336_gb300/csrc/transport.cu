// transport.cu -- the primaries: phase space, then the persistent, event-based stepping
// kernel (the secondary generations run in drain.cu).
//
// One lane carries one proton (Sec. II.B.1, one history per thread); when its
// proton stops, leaves the grid or is absorbed in a non-elastic collision, the
// lane takes the next sampled primary from a global counter (warp-aggregated), so
// warps stay full until the work runs out.  Per step (Sec. II.A.3):
//   step = min(lambda, d, R), random hinge with Highland x 1.07 deflection,
//   mean loss by range-table inversion (Eq. 2) plus Bohr straggling,
//   deposit to the step-start voxel as a 64-bit fixed-point atomic;
// nuclear elastic collisions (Sec. II.A.5) are handled in place, non-elastic
// ones (Sec. II.A.4) are appended to the event queue for the cascade kernel.
// Tables (ranges, inverse ranges, cross-sections) are staged in shared memory.
#include "transport_step.cuh"

namespace pmc {
namespace {

#ifndef PMC_TRANSPORT_MIN_BLOCKS
#define PMC_TRANSPORT_MIN_BLOCKS 3   // measured best on GB300: 3 resident blocks of 256 per SM
#endif

// Phase space of the primaries (Sec. II.B.2): spot sampling of work items w_begin..w_end-1,
// one thread per history, written to the generation's input queue as records the transport
// lanes take when they refill.  Sampling here, at full width, keeps two Philox blocks, the
// Box-Muller transforms and the spot search out of the transport kernel's refill, where
// they ran on the one or two lanes of a warp that had just finished a history.
__global__ void __launch_bounds__(256) phase_space_kernel(const TransportArgs a) {
  const unsigned long long n = a.w_end - a.w_begin;
  const unsigned long long seed = *a.seed;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  PrimaryRecord* out = reinterpret_cast<PrimaryRecord*>(a.qin);
  Acc acc;
  for (unsigned long long i = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    PState p;
    const bool alive = init_primary(a, key, a.w_begin + i, p, acc);
    out[i] = pack_primary(p, alive);
  }
  unsigned long long inc = static_cast<unsigned long long>(acc.inc), esc = static_cast<unsigned long long>(acc.esc);
  for (int o = 16; o > 0; o >>= 1) {
    inc += __shfl_xor_sync(0xffffffffu, inc, o);
    esc += __shfl_xor_sync(0xffffffffu, esc, o);
  }
  if ((threadIdx.x & 31u) == 0) {
    if (inc) atomicAdd(&a.cnt->incident, inc);
    if (esc) atomicAdd(&a.cnt->escaped, esc);
  }
}

template <bool kLet, bool kMol, bool kVav, int kMinBlocks>
__global__ void __launch_bounds__(256, kMinBlocks) transport_kernel(const TransportArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned long long n_items = a.w_end - a.w_begin;
  if (n_items == 0) return;
  if (static_cast<unsigned long long>(blockIdx.x) * blockDim.x >= n_items) return;

  const StagedTables tb = stage_transport_tables<kMol>(a, smem);
  const Physics& ph = *tb.ph;
  const float2 *rt = tb.rt, *et = tb.et;
  const float* st = tb.st;
  const float4* mol = tb.mol;
  GlobalQueues q{a};

  const unsigned long long seed = *a.seed;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  const unsigned lane = threadIdx.x & 31u;
  PState p;
  bool alive = false, drained = false;
  Acc acc;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !alive && !drained);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned base = 0;
      if (static_cast<int>(lane) == leader) base = atomicAdd(a.work, static_cast<unsigned>(__popc(need)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!alive && !drained) {
        const unsigned long long idx = base + __popc(need & ((1u << lane) - 1u));
        if (idx < n_items) {
          alive = load_primary(reinterpret_cast<const PrimaryRecord*>(a.qin)[idx], p);
        } else {
          drained = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, !alive && drained)) break;
    if (alive) alive = step<kLet, kMol, kVav>(a, ph, rt, et, st, mol, key, p, acc, q);
  }

  flush_transport_counters(acc, a.cnt, true);
}

}  // namespace

size_t transport_smem_bytes(int n_cls, int n_mat, bool moliere) {
  const size_t b = (sizeof(Physics) + 15) / 16 * 16 + 1ull * n_cls * (kNE + kNR) * sizeof(float2) +
                   1ull * n_mat * kNS * sizeof(float);
  return moliere ? (b + 15) / 16 * 16 + moliere_table_bytes(n_mat) : b;
}

namespace {
// the specialisations: (LET scored) + 2 (Moliere) + 4 (Vavilov)
constexpr int kP = PMC_TRANSPORT_MIN_BLOCKS;
void (*const kTransportKernels[8])(const TransportArgs) = {
    transport_kernel<false, false, false, kP>, transport_kernel<true, false, false, kP>,
    transport_kernel<false, true, false, kP>,  transport_kernel<true, true, false, kP>,
    transport_kernel<false, false, true, kP>,  transport_kernel<true, false, true, kP>,
    transport_kernel<false, true, true, kP>,   transport_kernel<true, true, true, kP>};
}  // namespace

cudaError_t transport_occupancy(int block, size_t smem, int* blocks) {
  int lo = 1 << 30;
  for (int i = 0; i < 8; ++i) {
    const auto k = kTransportKernels[i];
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, block, smem);
    if (e != cudaSuccess) return e;
    lo = b < lo ? b : lo;
  }
  *blocks = lo;
  return cudaSuccess;
}

cudaError_t launch_transport(const TransportArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  // the debug deposit log runs the paper's physics options only (Highland, Bohr, no LET)
  if (a.dlog && (a.let_num || a.mol || a.vav)) return cudaErrorInvalidValue;
  // the primaries are sampled into the generation's (otherwise unused) input queue first
  const unsigned long long n = a.w_end - a.w_begin;
  if (!a.qin || n > a.qin_cap) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  const unsigned long long blocks = (n + 255) / 256;
  phase_space_kernel<<<static_cast<unsigned>(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kTransportKernels[(a.let_num ? 1 : 0) + (a.mol ? 2 : 0) + (a.vav ? 4 : 0)]<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pmc
