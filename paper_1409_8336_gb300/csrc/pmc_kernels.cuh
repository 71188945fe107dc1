// pmc_kernels.cuh -- kernel argument blocks and launch wrappers of the engine.
#pragma once

#include "pmc_device.cuh"

namespace pmc {

struct Geometry {
  int nx, ny, nz;
  float dx, dy, dz, x0, y0, z0, idx, idy, idz;
  const uint8_t* mat;              // per voxel material (or NULL when hu is used)
  const float* rho;                // per voxel density
  const int16_t* hu;               // per voxel HU (or NULL)
};

// A spot in work order (highest energy first), with the first history index
// it owns and its offset in the work order.
struct SpotDev {
  float E, sE, x, y, sx, sy, u, v, w, pad0;
  unsigned long long h_first, w_first;
};

// One logged deposit (the debug deposit log): the tally entry (voxel, group) received
// llrint(e[0] 2^24) - llrint(e[1] 2^24) - llrint(e[2] 2^24) units of 2^-24 MeV.
struct DepositRecord {
  int voxel, group;
  double e[3];
};
static_assert(sizeof(DepositRecord) == 32, "deposit record is 32 bytes");

__device__ __forceinline__ void log_deposit(DepositRecord* log, unsigned long long* count, unsigned long long cap,
                                            int v, unsigned b, double e0, double e1, double e2) {
  const unsigned long long i = atomicAdd(count, 1ull);
  if (i < cap) {
    DepositRecord r;
    r.voxel = v;
    r.group = static_cast<int>(b);
    r.e[0] = e0;
    r.e[1] = e1;
    r.e[2] = e2;
    log[i] = r;
  }
}

struct TransportArgs {
  const Physics* phys;
  const float2* rtab;              // [n_cls][kNE] range splines
  const float2* etab;              // [n_cls][kNR] inverse splines
  const float* stab;               // [n_mat][kNS] total cross-section per unit density
  const float4* mol;               // [kMolN] Moliere distribution functions, or NULL (Highland)
  const float* vav;                // Vavilov straggling table [kVavNB][kVavNK][kVavNU], or NULL (Bohr)
  Geometry g;
  unsigned long long* tally;       // [n_voxels][B]
  int B;
  const unsigned long long* seed;  // device scalar
  const SpotDev* spots;
  int n_spots;
  unsigned long long w_begin, w_end;   // the primaries of this launch, in work order
  Particle* qin;                   // their sampled states (PrimaryRecord, one per slot) [qin_cap]
  unsigned qin_cap;
  Particle* qsec;
  unsigned* qsec_count;
  unsigned qsec_cap;
  Particle* qne;
  unsigned* qne_count;
  unsigned qne_cap;
  unsigned* work;                  // work counter of this launch
  Counters* cnt;
  long long* hist;                 // per-history ledger [hist_n][4] or NULL
  unsigned long long hist_n;
  float* esc;                      // escape record [esc_cap][8] or NULL
  unsigned long long esc_cap;
  unsigned long long* let_num;     // [n_voxels][B] sum of q * LET (2^-24 MeV keV/um), or NULL
  unsigned long long* let_den;     // [n_voxels][B] sum of q over the same deposits (2^-24 MeV)
  DepositRecord* dlog;             // debug deposit log [dlog_cap], or NULL
  unsigned long long* dlog_count;
  unsigned long long dlog_cap;
};

// A residual nucleus handed from the cascade kernel to the evaporation kernel:
// the event, the residual's state, and where the event's random stream stands.
struct __align__(16) EvapRecord {
  Particle ev;                     // the event (position, direction, voxel, identity)
  float4 buf;                      // the stream's buffered uniforms
  double Ex, px, py, pz, bind;     // excitation, recoil momentum, binding so far (MeV)
  unsigned draw;                   // the stream's next Philox block
  int pos;                         // next uniform in buf
  int Z, A, k, retries;            // residual, products emitted so far, attempts redrawn
};
static_assert(sizeof(EvapRecord) == 128, "evaporation record is 128 bytes");

struct CascadeArgs {
  const NucleusModel* nuclei;      // [n_nuc]
  const float* btab;               // binding energies [kMaxZ][kMaxA], then A^(1/3)
  int n_nuc;
  Geometry g;
  unsigned long long* tally;
  int B;
  const unsigned long long* seed;
  const Particle* qne;
  const unsigned* qne_count;
  unsigned qne_cap;
  Particle* qsec;
  unsigned* qsec_count;
  unsigned qsec_cap;
  Counters* cnt;
  long long* hist;
  unsigned long long hist_n;
  EvapRecord* rec;                 // residuals for the evaporation kernel [rec_cap]
  unsigned* rec_count;
  unsigned rec_cap;
  unsigned* work;                  // event counter of the cascade kernel
  DepositRecord* dlog;             // debug deposit log [dlog_cap], or NULL
  unsigned long long* dlog_count;
  unsigned long long dlog_cap;
};

// Control block of a drain launch (device memory; the stamp survives from run to run, so
// the block and the ready flags are zeroed together once, when they are allocated).  Each
// counter that many warps update or poll has a 128-byte line of its own.
struct DrainCounter {
  unsigned v;
  unsigned pad[31];
};
struct DrainCtl {
  DrainCounter pq_tail, pq_head;   // particle queue: slots reserved by producers / taken by lanes
  DrainCounter eq_tail, eq_head;   // event queue: the same
  DrainCounter xq_tail, xq_head;   // residual nuclei waiting for their evaporation: the same
  DrainCounter completed;          // items finished (or dropped for want of room)
  unsigned pq_n0, eq_n0;           // slots written before the launch
  unsigned error;                  // a bounded wait ran out
  unsigned stamp;                  // this launch's ready mark
  unsigned pad[28];
};
static_assert(sizeof(DrainCtl) == 1024, "drain control block is eight 128-byte lines");

// The secondary generations of a sub-group in one launch: the transport and cascade
// argument blocks (their queue fields unused), the particle and event queues with a ready
// mark per slot, and where the items already queued are counted.
struct DrainArgs {
  TransportArgs t;
  CascadeArgs c;
  Particle* pq;                    // protons to transport [pq_cap]
  unsigned* pq_ready;
  unsigned pq_cap;
  const unsigned* pq_n0;           // protons queued before the launch
  Particle* eq;                    // non-elastic events [eq_cap]
  unsigned* eq_ready;
  unsigned eq_cap;
  const unsigned* eq_n0;           // events queued before the launch, or NULL
  EvapRecord* xq;                  // residual nuclei of finished cascades, to evaporate [xq_cap]
  unsigned* xq_ready;
  unsigned xq_cap;
  DrainCtl* ctl;
  unsigned phantom;                // items counted as queued that never come (debug: 0)
  int idle_limit;                  // polls of an idle warp before it gives up (0: the default)
};

struct StatsArgs {
  const unsigned long long* tally;
  int B;
  long long n_vox;
  Geometry g;
  const Physics* phys;
  double* dose;
  double* sigma;
  const unsigned long long* let_num;  // LET tallies or NULL
  const unsigned long long* let_den;
  double* let;                        // dose-averaged LET (keV/um) and its standard error
  double* let_sigma;
};

size_t transport_smem_bytes(int n_cls, int n_mat, bool moliere);
// The primaries w_begin..w_end-1: phase space into a.qin (capacity a.qin_cap), then transport.
cudaError_t launch_transport(const TransportArgs& a, int grid, int block, size_t smem, cudaStream_t s);
// Resident blocks per SM of the transport kernel.
cudaError_t transport_occupancy(int block, size_t smem, int* blocks);
// The cascade of the events in a.qne (persistent, lanes refilled from a.work) and the
// evaporation of their residuals (a.rec); a.work and a.rec_count must be zero.
cudaError_t launch_cascade(const CascadeArgs& a, cudaStream_t s);
cudaError_t launch_stats(const StatsArgs& a, cudaStream_t s);
// Shared memory, resident blocks per SM and launch of the drain (its control block is set up
// by a one-thread kernel launched first, on the same stream).
size_t drain_smem_bytes(int n_cls, int n_mat, bool moliere, int n_nuc);
cudaError_t drain_occupancy(int block, size_t smem, int* blocks);
cudaError_t launch_drain(const DrainArgs& d, int grid, int block, size_t smem, cudaStream_t s);

cudaError_t launch_surrogate_dataset(const NucleusModel* nuclei, const float* btab, const int* slot_nuc, int n_slots,
                                     unsigned long long seed, unsigned long long n, float* out, cudaStream_t s);

// C[m][n] (=|+=) sum_k A(m,k) B(k,n) (+ bias[n]) (ReLU) (* [mask[m][n] > 0]) with
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], FP32 in memory, BF16 operands on the
// 5th-generation tensor cores (tcgen05, 128-row tiles, FP32 accumulators in tensor memory); K is
// split over ws (room for ws_floats partial sums) when the tiles alone would leave SMs idle.  A
// tensor-core wait that ran out raises *err.
cudaError_t launch_gemm_tc(int M, int N, int K, const float* A, long long sam, long long sak, const float* B,
                          long long sbk, long long sbn, float* C, long long ldc, const float* bias, bool relu,
                          const float* mask, bool accumulate, float* ws, size_t ws_floats, int* err, int n_sm,
                          cudaStream_t s);
cudaError_t launch_mlp_rows(int rows, const float* X, const void* Wb, const float* P, float* Y, int* err, int n_sm,
                            bool check_waits, cudaStream_t s);
// The inference weights: BF16, each streamed chunk in the byte order of its shared-memory buffer.
size_t packed_weight_bytes();
cudaError_t launch_pack_weights(const float* P, void* packed, cudaStream_t s);
cudaError_t launch_pinball(int rows, const float* yhat, const float* y, const float* tau, const float* mask,
                           float* grad, float* loss, cudaStream_t s);
cudaError_t launch_colsum(int rows, int N, const float* G, float* db, cudaStream_t s);
cudaError_t launch_adamw(int n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                         float wd, int step, cudaStream_t s);
cudaError_t launch_train_rows(int batch, const float* feat, const unsigned* perm, unsigned long long first,
                              unsigned long long n_events, unsigned long long seed, unsigned step, float* X, float* Y,
                              float* tau, float* mask, cudaStream_t s);
cudaError_t launch_surrogate_events(const unsigned* n_ev, unsigned cap, const Particle* qne, const int* nuc_slot,
                                    const unsigned long long* seed, const void* Wb, const float* P,
                                    unsigned long long* tally, int B, Particle* qsec, unsigned* qsec_count,
                                    unsigned qsec_cap, Counters* cnt, long long* hist, unsigned long long hist_n,
                                    int grid, cudaStream_t s);

// Yields of a batch of non-elastic events (energies in 2^-24 MeV).
struct EventYields {
  unsigned long long events, transparent, retries;
  unsigned long long count[6];          // n, p, d, t, 3He, alpha emitted
  long long energy[6];                  // their kinetic energies
  long long residual, excitation, binding;
};

cudaError_t launch_inc_yields(const NucleusModel* nu, const float* btab, float E, unsigned long long seed,
                              unsigned long long pid0, unsigned long long n, EventYields* out, cudaStream_t s);

// Gamma plan in device memory: this head, then at kGammaHeadBytes the offsets of the
// search sphere sorted by their distance term.
struct GammaHead {
  unsigned long long n_eval, n_pass;  // written by each comparison
  unsigned long long max_key;         // max(ref) as an order-preserving integer
  unsigned long long work;            // next chunk of voxels to claim
  int n_off;                          // written by the plan
  int pad;
  double dx, dy, dz, dta, search;     // what the plan was made for (mm)
};
constexpr size_t kGammaHeadBytes = 256;
static_assert(sizeof(GammaHead) <= kGammaHeadBytes, "gamma head fits");

// One neighbour offset of the gamma search sphere: voxel steps and the distance
// term |r|^2 / dta^2 (FP64), 16 bytes.
struct alignas(16) GammaOffset {
  int16_t kx, ky, kz, pad;
  double r_term;
};
static_assert(sizeof(GammaOffset) == 16, "gamma offset layout");

cudaError_t launch_gamma(const double* ref, const double* ev, int nx, int ny, int nz, void* plan, double dose_pct,
                         double threshold, float* gamma, cudaStream_t s);

// debug entry points
cudaError_t launch_debug_philox(const uint4* ctr, uint2 key, uint4* out, int n, cudaStream_t s);
cudaError_t launch_debug_tables(const Physics* ph, const float2* rt, const float2* et, int cls, const double* E,
                                double* r, double* e, int n, cudaStream_t s);
cudaError_t launch_debug_inc(const NucleusModel* nu, const float* btab, float E, unsigned long long seed,
                             unsigned long long pid0, int n, double* summary, double* products, int cap,
                             cudaStream_t s);
cudaError_t launch_debug_elastic(const Physics* ph, int nuclide, float E, const double* u, double* out, int n,
                                 cudaStream_t s);

__device__ __forceinline__ void voxel_props(const Physics& ph, const Geometry& g, int v, int& m, float& rho) {
  if (g.hu) {
    const int h = g.hu[v];
    int b = ph.n_hu - 1;
    for (int k = 0; k < ph.n_hu; ++k) {
      if (h >= ph.hu[k].lo && h < ph.hu[k].hi) { b = k; break; }
    }
    if (h < ph.hu[0].lo) b = 0;
    m = ph.hu[b].mat;
    rho = ph.hu[b].a + ph.hu[b].b * static_cast<float>(h);
  } else {
    m = g.mat[v];
    rho = g.rho[v];
  }
}

}  // namespace pmc
