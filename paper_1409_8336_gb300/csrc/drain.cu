// drain.cu -- the secondary generations of a sub-group in one persistent launch (Sec. II.B.2:
// the secondary protons and the non-elastic events they cause, until none is left).
//
// After the primaries and the cascades of their events, a sub-group leaves a few 1e5
// secondary protons, which cause a few 1e4 further events over a handful of generations.
// Launched generation by generation, each transport and each cascade launch lasts as long as
// its longest track or cascade while most of the GPU idles, and the generations add up.  Here
// lanes take what is ready from three global queues -- protons to step on five SMs in six;
// events to run through the cascade, and the residual nuclei those leave, to evaporate, on the
// sixth -- and what an item produces goes back to them, so the long tracks and long cascades of
// different lineages overlap.  The launch ends when every item ever queued has been finished.
//
// Queues: a producer reserves a slot by an atomic add on the tail, writes it and marks it
// ready with this launch's stamp (release).  Lanes take slots by an atomic add on the head
// (a claim never fails, so thousands of warps claiming at once do not serialise on a
// compare-and-swap); a slot taken ahead of the tail is a ticket for an item not yet produced,
// which the lane checks once per iteration on the slot's own ready mark (acquire) while the
// rest of its warp works.  The launch is done when the items finished (or dropped for want of
// room) equal the items ever queued (the two tails): an item is counted finished only after
// everything it produced has been queued.  Every wait is bounded; one that runs out marks the
// launch's error, counts an error for the run (PMC_E_TIMEOUT on the host) and ends it.
//
// Each item's result depends only on its identity (the random numbers are keyed by it), so
// the tallies do not depend on which lane takes what, or when: the run is bit-reproducible.
#include "transport_step.cuh"
#include "cascade_event.cuh"

namespace pmc {
namespace {

constexpr int kIdlePolls = 1 << 20;      // iterations of a warp with nothing to do (a few seconds)

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Appends r: false (nothing queued; counted finished at once) when the queue is full.
__device__ __forceinline__ bool drain_push(Particle* q, unsigned* ready, unsigned cap, unsigned* tail, DrainCtl* ctl,
                                           unsigned stamp, const Particle& r) {
  const unsigned i = atomicAdd(tail, 1u);
  if (i >= cap) {
    atomicAdd(&ctl->completed.v, 1u);
    return false;
  }
  q[i] = r;
  st_release(ready + i, stamp);
  return true;
}

// Takes up to `want` slots of a queue when its tail is ahead of its head: the first slot,
// how many (0 when the queue looks empty).  Some may lie ahead of the tail (tickets).
__device__ __forceinline__ unsigned drain_take(unsigned* head, const unsigned* tail, unsigned cap, unsigned want,
                                               unsigned& base) {
  const unsigned h = ld_relaxed(head);
  const unsigned t = min(ld_relaxed(tail), cap);
  if (h >= t) return 0;
  const unsigned k = min(want, t - h);
  base = atomicAdd(head, k);
  return k;
}

// Appends a residual nucleus for evaporation: false (nothing queued) when the queue is full.
__device__ __forceinline__ bool drain_push_residual(const DrainArgs& d, unsigned stamp, const EvapRecord& r) {
  const unsigned i = atomicAdd(&d.ctl->xq_tail.v, 1u);
  if (i >= d.xq_cap) {
    atomicAdd(&d.ctl->completed.v, 1u);
    return false;
  }
  d.xq[i] = r;
  st_release(d.xq_ready + i, stamp);
  return true;
}

// Queue policy of the transport step inside the drain.
struct DrainQueues {
  const DrainArgs& d;
  unsigned stamp;
  __device__ __forceinline__ bool event(const Particle& r) const {
    return drain_push(d.eq, d.eq_ready, d.eq_cap, &d.ctl->eq_tail.v, d.ctl, stamp, r);
  }
  __device__ __forceinline__ bool secondary(const Particle& r) const {
    return drain_push(d.pq, d.pq_ready, d.pq_cap, &d.ctl->pq_tail.v, d.ctl, stamp, r);
  }
};

// Environment of the event sink inside the drain: protons emitted by cascades and
// evaporation go to the particle queue.
struct DrainEnv {
  const DrainArgs* d;
  unsigned stamp;
  __device__ __forceinline__ unsigned long long* tally() const { return d->c.tally; }
  __device__ __forceinline__ int B() const { return d->c.B; }
  __device__ __forceinline__ long long* hist() const { return d->c.hist; }
  __device__ __forceinline__ unsigned long long hist_n() const { return d->c.hist_n; }
  __device__ __forceinline__ DepositRecord* dlog() const { return d->c.dlog; }
  __device__ __forceinline__ unsigned long long* dlog_count() const { return d->c.dlog_count; }
  __device__ __forceinline__ unsigned long long dlog_cap() const { return d->c.dlog_cap; }
  __device__ __forceinline__ bool push(const Particle& r) const {
    return drain_push(d->pq, d->pq_ready, d->pq_cap, &d->ctl->pq_tail.v, d->ctl, stamp, r);
  }
};

// One lane's event: the cascade's steps in the order the sequential event routine takes
// them (so the event's random stream is consumed identically), one per iteration; the
// residual nucleus, with the position of the stream, is then queued for its evaporation.
// (Evaporated in place, a lane's chain of tens of microseconds held up the cascades of the
// other 31 lanes of its warp, one finishing lane after another; queued, residuals are
// evaporated by warps that take 32 of them at once, as the evaporation kernel does.)
struct LaneEvent {
  Stream st;
  IncState s;
  const NucleusModel* nu;
  int attempt, retries;
  bool setup;
};

// Advances the lane's event by one step; true when the event is finished.
__device__ __forceinline__ bool event_step(LaneEvent& e, IncP* P, const float* bt, EventSink<DrainEnv>& sk) {
  if (e.setup) {
    inc_setup(*e.nu, sk.ev.E, e.st, P, e.s);
    e.setup = false;
    return false;
  }
  if (!inc_flight(*e.nu, e.st, P, e.s)) return false;
  P[e.s.ip] = e.s.p;
  if (++e.s.ip < e.s.n) {
    e.s.p = P[e.s.ip];
    e.s.crossings = 0;
    e.s.iters = 0;
    return false;
  }
  Residual r;
  if (!inc_residual(*e.nu, bt, sk.ev.E, P, e.s, r)) {
    ++e.retries;
    if (++e.attempt < kIncRetries) {
      e.setup = true;
      return false;
    }
    sk.transparent(e.retries);
    return true;
  }
  const int k = inc_emit(P, e.s.n, sk);
  EvapRecord x;
  x.ev = sk.ev;
  x.Ex = r.Ex; x.px = r.px; x.py = r.py; x.pz = r.pz; x.bind = r.bind;
  x.buf = e.st.buf; x.draw = e.st.draw; x.pos = e.st.pos;
  x.Z = r.Z; x.A = r.A; x.k = k; x.retries = e.retries;
  if (!drain_push_residual(*sk.env.d, sk.env.stamp, x)) evaporate(bt, e.st, r, k, e.retries, sk);   // no room
  return true;
}

// The evaporation of a queued residual nucleus (its random stream resumes where the cascade
// left it).
__device__ __forceinline__ void evaporate_record(const EvapRecord& x, const float* bt, int B,
                                                 EventSink<DrainEnv>& sk) {
  sk.ev = x.ev;
  sk.b = x.ev.root % static_cast<unsigned>(B);
  Stream st{sk.key, x.ev.pid, x.draw, x.pos, x.buf};
  Residual r;
  r.Ex = x.Ex; r.px = x.px; r.py = x.py; r.pz = x.pz; r.bind = x.bind; r.Z = x.Z; r.A = x.A;
  evaporate(bt, st, r, x.k, x.retries, sk);
}

__global__ void drain_init_kernel(DrainCtl* ctl, const unsigned* pq_n0, unsigned pq_cap, const unsigned* eq_n0,
                                  unsigned eq_cap) {
  const unsigned p0 = min(*pq_n0, pq_cap), e0 = eq_n0 ? min(*eq_n0, eq_cap) : 0u;
  ctl->pq_tail.v = p0;
  ctl->pq_head.v = 0;
  ctl->eq_tail.v = e0;
  ctl->eq_head.v = 0;
  ctl->xq_tail.v = 0;
  ctl->xq_head.v = 0;
  ctl->completed.v = 0;
  ctl->pq_n0 = p0;
  ctl->eq_n0 = e0;
  ctl->error = 0;
  ctl->stamp = ctl->stamp + 1u;
}

// SM roles: the blocks on one SM in kEventSm take events, those on the others protons, so that
// no SM runs both the cascade and the transport code, whose instructions together overflow an
// SM's instruction caches (measured on the slab workload, drain per transport: every lane
// taking either kind 1.76 ms; one SM in 3, 4, 6, 8, 12 for events: 1.42, 1.58, 1.31, 1.60, 1.63
// ms; with the residual queue, one in 4, 5, 6, 8: 1.43, 1.24, 1.23-1.25, 1.46 ms).  A warp
// idle for kRoleFallback polls takes either kind: the other kind's SMs may hold no block of
// this launch (another launch occupying them).
constexpr unsigned kEventSm = 6;
constexpr int kRoleFallback = 2048;
// two blocks of 256 per SM (128 registers); with three (85) the spills cost 1.7x
template <bool kLet, bool kMol, bool kVav>
__global__ void __launch_bounds__(256, 2) drain_kernel(const DrainArgs d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TransportArgs& a = d.t;
  const StagedTables tb = stage_transport_tables<kMol>(a, smem);
  NucleusModel* nuc = reinterpret_cast<NucleusModel*>(tb.end);
  float* bt = reinterpret_cast<float*>(nuc + d.c.n_nuc);
  {
    const float* src = reinterpret_cast<const float*>(d.c.nuclei);
    float* dst = reinterpret_cast<float*>(nuc);
    const int nw = d.c.n_nuc * static_cast<int>(sizeof(NucleusModel) / 4);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < kBtabFloats; i += blockDim.x) bt[i] = d.c.btab[i];
  }
  __syncthreads();
  const Physics& ph = *tb.ph;
  DrainCtl* ctl = d.ctl;
  const unsigned stamp = ld_relaxed(&ctl->stamp);
  const unsigned pq_n0 = ld_relaxed(&ctl->pq_n0), eq_n0 = ld_relaxed(&ctl->eq_n0);
  const unsigned long long seed = *a.seed;
  const uint2 key = make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32));
  const unsigned lane = threadIdx.x & 31u;
  DrainQueues q{d, stamp};
  EventSink<DrainEnv> sk;
  sk.env = DrainEnv{&d, stamp};
  sk.key = key;
  sk.dep = sk.esc = sk.bnd = 0;
  sk.sec = sk.dropped = sk.retries = sk.n_transparent = 0;
  PState p;
  Acc acc;
  IncP P[kIncStack];
  LaneEvent ev;
  ev.nu = nuc;
  // 0: idle, 1: a proton in hand, 2: an event in hand, 5: a residual nucleus to evaporate;
  // 3 / 4 / 6: a ticket for a proton / event / residual slot not yet written
  int role = 0;
  unsigned slot = 0;
  int polls = 0, backoff = 0, skip = 0, nap = 128, idle_run = 0;
  unsigned smid;
  asm("mov.u32 %0, %%smid;" : "=r"(smid));
  const bool event_sm = smid % kEventSm == 0;
  // takes the item of a written slot of queue `kind` (0 protons, 1 events, 2 residuals);
  // false for an invalid event
  auto take = [&](int kind, unsigned i) {
    if (kind == 1) {
      const Particle r = d.eq[i];
      if (r.target < 0 || r.target >= d.c.n_nuc) return false;
      sk.ev = r;
      sk.b = r.root % static_cast<unsigned>(a.B);
      ev.st = Stream{key, r.pid, 0u, 4, make_float4(0.f, 0.f, 0.f, 0.f)};
      ev.nu = nuc + r.target;
      ev.attempt = 0;
      ev.retries = 0;
      ev.setup = true;
      role = 2;
    } else if (kind == 2) {
      slot = i;
      role = 5;
    } else {
      init_queued(a, key, d.pq[i], p);
      role = 1;
    }
    return true;
  };
  auto finish = [&]() {   // the item in hand is done, with everything it produced queued
    role = 0;
    __threadfence();
    atomicAdd(&ctl->completed.v, 1u);
  };
  for (;;) {
    // tickets: is the slot written yet?
    if (role == 3 || role == 4 || role == 6) {
      const int kind = role == 3 ? 0 : (role == 4 ? 1 : 2);
      const unsigned* ready = kind == 0 ? d.pq_ready : (kind == 1 ? d.eq_ready : d.xq_ready);
      if (ld_acquire(ready + slot) == stamp) {
        if (!take(kind, slot)) {
          atomicExch(&ctl->error, 1u);
          acc.errors++;
          finish();
        }
      }
    }
    const unsigned idle = __ballot_sync(0xffffffffu, role == 0);
    const unsigned busy = __ballot_sync(0xffffffffu, role == 1 || role == 2 || role == 5);
    // A warp that still holds work and found the queues empty looks again only after a few
    // steps (up to 16): the claim's loads would otherwise lengthen every step of its tracks.
    bool look = idle != 0u;
    if (look && busy && skip > 0) {
      --skip;
      look = false;
    }
    if (look) {
      // Claims for the idle lanes, by the SM's role (after a long idle spell any kind).  An
      // event SM's warp that holds no cascade takes residual nuclei first, and then nothing
      // else that round, so that its lanes evaporate together; otherwise events.  A proton
      // SM's warp takes protons.
      const bool holds_inc = __ballot_sync(0xffffffffu, role == 2 || role == 4) != 0u;
      const int leader = __ffs(idle) - 1;
      unsigned b0 = 0, n0 = 0, b1 = 0, n1 = 0, b2 = 0, n2 = 0;
      const bool any = idle_run >= kRoleFallback;
      if (static_cast<int>(lane) == leader) {
        const unsigned want = __popc(idle);
        if ((event_sm || any) && !holds_inc) n2 = drain_take(&ctl->xq_head.v, &ctl->xq_tail.v, d.xq_cap, want, b2);
        if ((event_sm || any) && n2 == 0) n1 = drain_take(&ctl->eq_head.v, &ctl->eq_tail.v, d.eq_cap, want, b1);
        if ((!event_sm || any) && n1 + n2 < want)
          n0 = drain_take(&ctl->pq_head.v, &ctl->pq_tail.v, d.pq_cap, want - n1 - n2, b0);
      }
      b0 = __shfl_sync(0xffffffffu, b0, leader);
      n0 = __shfl_sync(0xffffffffu, n0, leader);
      b1 = __shfl_sync(0xffffffffu, b1, leader);
      n1 = __shfl_sync(0xffffffffu, n1, leader);
      b2 = __shfl_sync(0xffffffffu, b2, leader);
      n2 = __shfl_sync(0xffffffffu, n2, leader);
      if (role == 0) {
        const unsigned r = __popc(idle & ((1u << lane) - 1u));
        if (r < n0 + n1 + n2) {
          const int kind = r < n2 ? 2 : (r < n2 + n1 ? 1 : 0);
          const unsigned i = kind == 2 ? b2 + r : (kind == 1 ? b1 + (r - n2) : b0 + (r - n2 - n1));
          const unsigned cap = kind == 0 ? d.pq_cap : (kind == 1 ? d.eq_cap : d.xq_cap);
          const unsigned* ready = kind == 0 ? d.pq_ready : (kind == 1 ? d.eq_ready : d.xq_ready);
          const unsigned nb = kind == 0 ? pq_n0 : (kind == 1 ? eq_n0 : 0u);
          if (i < cap) {   // a slot at or beyond the capacity can never be written: none taken
            if (!(i < nb || ld_acquire(ready + i) == stamp)) {
              role = kind == 0 ? 3 : (kind == 1 ? 4 : 6);
              slot = i;
            } else if (!take(kind, i)) {
              atomicExch(&ctl->error, 1u);
              acc.errors++;
              finish();
            }
          }
        }
      }
      if (n0 + n1 + n2 > 0) {
        backoff = 0;
      } else if (busy) {
        backoff = min(2 * backoff + 1, 15);
        skip = backoff;
      }
    }
    if (__ballot_sync(0xffffffffu, role == 1 || role == 2 || role == 5) == 0u) {
      // nothing in hand: done, stopped, or waiting for work.  The decision is lane 0's,
      // broadcast, so that the whole warp leaves the loop together (the counter flush after it
      // uses full-warp shuffles).  Done: every item ever queued is finished (read the finished
      // count first: an item queued after that read makes the tails larger, never equal).
      unsigned stop = 0;
      if (lane == 0) {
        const unsigned fin = ld_acquire(&ctl->completed.v);
        const unsigned pushed = ld_relaxed(&ctl->pq_tail.v) + ld_relaxed(&ctl->eq_tail.v) +
                                ld_relaxed(&ctl->xq_tail.v) + d.phantom;
        stop = (fin == pushed || ld_relaxed(&ctl->error) != 0u) ? 1u : 0u;
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) break;
      if (++polls > (d.idle_limit > 0 ? d.idle_limit : kIdlePolls)) {
        if (lane == 0) {
          atomicExch(&ctl->error, 1u);
          acc.errors++;
        }
        break;
      }
      ++idle_run;
      __nanosleep(nap);
      nap = min(2 * nap, 4096);
      continue;
    }
    nap = 128;
    idle_run = 0;
    if (role == 1) {
      if (!step<kLet, kMol, kVav>(a, ph, tb.rt, tb.et, tb.st, tb.mol, key, p, acc, q)) finish();
    } else if (role == 2) {
      if (event_step(ev, P, bt, sk)) finish();
    } else if (role == 5) {
      evaporate_record(d.xq[slot], bt, a.B, sk);
      finish();
    }
  }
  flush_transport_counters(acc, a.cnt, false);
  flush_counters(sk, a.cnt);
}

template <bool kLet, bool kMol, bool kVav>
constexpr auto kDrain = drain_kernel<kLet, kMol, kVav>;
// [(LET scored) + 2 (Moliere) + 4 (Vavilov)], as for the transport kernel
void (*const kDrainKernels[8])(const DrainArgs) = {
    kDrain<false, false, false>, kDrain<true, false, false>, kDrain<false, true, false>, kDrain<true, true, false>,
    kDrain<false, false, true>,  kDrain<true, false, true>,  kDrain<false, true, true>,  kDrain<true, true, true>};

}  // namespace

size_t drain_smem_bytes(int n_cls, int n_mat, bool moliere, int n_nuc) {
  return (transport_smem_bytes(n_cls, n_mat, moliere) + 15) / 16 * 16 + static_cast<size_t>(n_nuc) * sizeof(NucleusModel) +
         kBtabFloats * sizeof(float);
}

cudaError_t drain_occupancy(int block, size_t smem, int* blocks) {
  int lo = 1 << 30;
  for (int i = 0; i < 8; ++i) {
    cudaError_t e = cudaFuncSetAttribute(kDrainKernels[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kDrainKernels[i], block, smem);
    if (e != cudaSuccess) return e;
    lo = b < lo ? b : lo;
  }
  *blocks = lo;
  return cudaSuccess;
}

cudaError_t launch_drain(const DrainArgs& d, int grid, int block, size_t smem, cudaStream_t s) {
  if (!d.pq || !d.eq || !d.xq || !d.pq_ready || !d.eq_ready || !d.xq_ready || !d.ctl || !d.pq_n0)
    return cudaErrorInvalidValue;
  if (d.t.dlog && (d.t.let_num || d.t.mol || d.t.vav)) return cudaErrorInvalidValue;
  drain_init_kernel<<<1, 1, 0, s>>>(d.ctl, d.pq_n0, d.pq_cap, d.eq_n0, d.eq_cap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kDrainKernels[(d.t.let_num ? 1 : 0) + (d.t.mol ? 2 : 0) + (d.t.vav ? 4 : 0)]<<<grid, block, smem, s>>>(d);
  return cudaGetLastError();
}

}  // namespace pmc
