// transport.cu -- persistent, event-based proton stepping kernel.
//
// One lane carries one proton (Sec. II.B.1, one history per thread); when its
// proton stops, leaves the grid or is absorbed in a non-elastic collision, the
// lane takes the next work item from a global counter (warp-aggregated), so
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
// Secondary generations hold few particles and last as long as their longest track: there a
// step's latency counts more than the number of resident warps, and with 2 blocks per SM the
// step has the registers to be shorter (secondary stage 1.50 against 1.61 ms on the slab).
#ifndef PMC_TRANSPORT_MIN_BLOCKS_SECONDARY
#define PMC_TRANSPORT_MIN_BLOCKS_SECONDARY 2
#endif

template <bool kLet, bool kMol, bool kVav, int kMinBlocks, bool kLog = false>
__global__ void __launch_bounds__(256, kMinBlocks) transport_kernel(const TransportArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned long long n_items =
      a.source == 0 ? (a.w_end - a.w_begin) : static_cast<unsigned long long>(min(*a.qin_count, a.qin_cap));
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
          if (a.source == 0) {
            alive = init_primary(a, key, a.w_begin + idx, p, acc);
          } else {
            init_queued(a, key, a.qin[idx], p);
            alive = true;
          }
        } else {
          drained = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, !alive && drained)) break;
    if (alive) alive = step<kLet, kMol, kVav, kLog>(a, ph, rt, et, st, mol, key, p, acc, q);
  }

  // flush the lane counters (warp reduction, one atomic per warp and counter)
  auto wsum = [](unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  const unsigned long long inc = wsum(static_cast<unsigned long long>(acc.inc));
  const unsigned long long dep = wsum(static_cast<unsigned long long>(acc.dep));
  const unsigned long long esc = wsum(static_cast<unsigned long long>(acc.esc));
  const unsigned long long steps = wsum(acc.steps), el = wsum(acc.el), inel = wsum(acc.inel);
  const unsigned long long sec = wsum(acc.sec), dropped = wsum(acc.dropped), errors = wsum(acc.errors);
  if (lane == 0) {
    Counters* c = a.cnt;
    if (inc) atomicAdd(&c->incident, inc);
    if (dep) atomicAdd(&c->deposited, dep);
    if (esc) atomicAdd(&c->escaped, esc);
    if (steps) atomicAdd(&c->steps, steps);
    if (steps && a.source == 0) atomicAdd(&c->steps_primary, steps);
    if (el) atomicAdd(&c->elastic, el);
    if (inel) atomicAdd(&c->inelastic, inel);
    if (sec) atomicAdd(&c->secondaries, sec);
    if (dropped) atomicAdd(&c->dropped, dropped);
    if (errors) atomicAdd(&c->errors, errors);
  }
}

}  // namespace

size_t transport_smem_bytes(int n_cls, int n_mat, bool moliere) {
  const size_t b = (sizeof(Physics) + 15) / 16 * 16 + 1ull * n_cls * (kNE + kNR) * sizeof(float2) +
                   1ull * n_mat * kNS * sizeof(float);
  return moliere ? (b + 15) / 16 * 16 + moliere_table_bytes(n_mat) : b;
}

namespace {
// the specialisations: [primaries, secondaries][(LET scored) + 2 (Moliere) + 4 (Vavilov)]
constexpr int kP = PMC_TRANSPORT_MIN_BLOCKS, kS = PMC_TRANSPORT_MIN_BLOCKS_SECONDARY;
template <int kB>
constexpr void (*kFamily[8])(const TransportArgs) = {
    transport_kernel<false, false, false, kB>, transport_kernel<true, false, false, kB>,
    transport_kernel<false, true, false, kB>,  transport_kernel<true, true, false, kB>,
    transport_kernel<false, false, true, kB>,  transport_kernel<true, false, true, kB>,
    transport_kernel<false, true, true, kB>,   transport_kernel<true, true, true, kB>};
void (*const* const kTransportKernels[2])(const TransportArgs) = {kFamily<kP>, kFamily<kS>};
// the debug deposit log, with the paper's physics options (Highland, Bohr, no LET)
void (*const kTransportLogKernels[2])(const TransportArgs) = {transport_kernel<false, false, false, kP, true>,
                                                              transport_kernel<false, false, false, kS, true>};
}  // namespace

cudaError_t transport_occupancy(int block, size_t smem, int* blocks_primary, int* blocks_secondary) {
  for (int g = 0; g < 2; ++g) {
    int lo = 1 << 30;
    for (int i = 0; i < 8; ++i) {
      const auto k = kTransportKernels[g][i];
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      int b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, block, smem);
      if (e != cudaSuccess) return e;
      lo = b < lo ? b : lo;
    }
    cudaError_t e = cudaFuncSetAttribute(kTransportLogKernels[g], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    *(g ? blocks_secondary : blocks_primary) = lo;
  }
  return cudaSuccess;
}

cudaError_t launch_transport(const TransportArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  if (a.dlog) {
    if (a.let_num || a.mol || a.vav) return cudaErrorInvalidValue;   // the log runs the default physics only
    kTransportLogKernels[a.source ? 1 : 0]<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  }
  kTransportKernels[a.source ? 1 : 0][(a.let_num ? 1 : 0) + (a.mol ? 2 : 0) + (a.vav ? 4 : 0)]<<<grid, block, smem, s>>>(
      a);
  return cudaGetLastError();
}

}  // namespace pmc
