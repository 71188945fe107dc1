// transport_step.cuh -- the condensed-history step of one proton (Sec. II.A.3) and what it
// needs: particle state, birth of primaries and queued particles, fixed-point deposits.
// Where a step hands on a non-elastic event or an elastic recoil proton is a policy (the
// generation kernel of transport.cu appends to global queues).
#pragma once

#include "pmc_kernels.cuh"

namespace pmc {
namespace {

struct PState {
  float x, y, z, u, v, w, E, nmfp;
  long long fE;        // fix(E), carried from step to step (a step's deposit is fE - fix(E1))
  int ix, iy, iz;
  unsigned k;          // step counter of this particle
  unsigned root;       // primary history
  unsigned b;          // statistical group
  unsigned long long pid;
};

struct Acc {           // per-lane counters flushed once at the end
  long long inc = 0, dep = 0, esc = 0;
  unsigned long long steps = 0, el = 0, inel = 0, sec = 0, dropped = 0, errors = 0;
};

// sin and cos of 2 pi u, u in [0, 1] (the azimuths and Box-Muller angles of a step).  The
// -use_fast_math build takes the special-function unit's approximations on [-pi, pi] (absolute
// error ~2^-21; 2 pi u = pi + t with both signs flipped), a few instructions against the ~25
// of the exactly reduced sincospi; the IEEE build keeps sincospi.
__device__ __forceinline__ void sincos_2pi(float u, float* sn, float* cs) {
#ifdef __USE_FAST_MATH__
  float a, b;
  __sincosf(6.28318531f * (u - 0.5f), &a, &b);
  *sn = -a;
  *cs = -b;
#else
  sincospif(2.0f * u, sn, cs);
#endif
}

__device__ __forceinline__ int vindex(const Geometry& g, int ix, int iy, int iz) {
  return (iz * g.ny + iy) * g.nx + ix;
}

// Distance from p along d to the faces of voxel (ix, iy, iz); axis of exit.
__device__ __forceinline__ float voxel_exit(const Geometry& g, float px, float py, float pz, float u, float v,
                                            float w, int ix, int iy, int iz, int& axis) {
  float best = 3.0e38f;
  axis = 0;
  if (u != 0.0f) {
    const float f = g.x0 + static_cast<float>(u > 0.0f ? ix + 1 : ix) * g.dx;
    const float s = fmaxf((f - px) / u, 0.0f);
    best = s;
  }
  if (v != 0.0f) {
    const float f = g.y0 + static_cast<float>(v > 0.0f ? iy + 1 : iy) * g.dy;
    const float s = fmaxf((f - py) / v, 0.0f);
    if (s < best) { best = s; axis = 1; }
  }
  if (w != 0.0f) {
    const float f = g.z0 + static_cast<float>(w > 0.0f ? iz + 1 : iz) * g.dz;
    const float s = fmaxf((f - pz) / w, 0.0f);
    if (s < best) { best = s; axis = 2; }
  }
  return best;
}

__device__ __forceinline__ void deposit(const TransportArgs& a, int v, const PState& p, long long q, Acc& acc) {
  atomicAdd(a.tally + static_cast<size_t>(v) * a.B + p.b, static_cast<unsigned long long>(q));
  acc.dep += q;
  if (a.hist && p.root < a.hist_n) atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + 4ull * p.root + 1),
                                             static_cast<unsigned long long>(q));
}

// Dose-averaged LET (Sec. IV): an energy loss q of the transported proton, weighted by
// L, the mean stopping power of the local medium over the path that lost it (keV/um).
__device__ __forceinline__ void score_let(const TransportArgs& a, int v, const PState& p, long long q, float L) {
  const size_t i = static_cast<size_t>(v) * a.B + p.b;
  atomicAdd(a.let_den + i, static_cast<unsigned long long>(q));
  atomicAdd(a.let_num + i, static_cast<unsigned long long>(__float2ll_rn(static_cast<float>(q) * L)));
}

__device__ __forceinline__ void escape(const TransportArgs& a, const PState& p, long long q, Acc& acc) {
  acc.esc += q;
  if (a.hist && p.root < a.hist_n) atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + 4ull * p.root + 2),
                                             static_cast<unsigned long long>(q));
}

__device__ __forceinline__ bool push(Particle* q, unsigned* count, unsigned cap, const Particle& r) {
  const unsigned i = atomicAdd(count, 1u);
  if (i >= cap) return false;
  q[i] = r;
  return true;
}

// Birth of primary work item wi: spot sampling (Sec. II.B.2, phase-space kernel).
__device__ __forceinline__ bool init_primary(const TransportArgs& a, uint2 key, unsigned long long wi, PState& p,
                                             Acc& acc) {
  int lo = 0, hi = a.n_spots;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.spots[mid].w_first <= wi) lo = mid; else hi = mid;
  }
  const SpotDev s = a.spots[lo];
  const unsigned long long h = s.h_first + (wi - s.w_first);
  const float4 r0 = draw4(key, h, 0u, 4u);
  const float rr = sqrtf(-2.0f * logf(r0.x));
  float sn, cs;
  sincospif(2.0f * r0.y, &sn, &cs);
  p.x = s.x + s.sx * rr * cs;
  p.y = s.y + s.sy * rr * sn;
  p.z = a.g.z0;
  p.E = fmaxf(s.E + s.sE * sqrtf(-2.0f * logf(r0.z)) * cospif(2.0f * r0.w), 0.0f);
  p.u = s.u; p.v = s.v; p.w = s.w;
  p.nmfp = -logf(draw4(key, h, 1u, 4u).x);
  p.pid = h;
  p.root = static_cast<unsigned>(h);
  p.b = static_cast<unsigned>(h % static_cast<unsigned long long>(a.B));
  p.k = 0;
  const long long q = fix(p.E);
  acc.inc += q;
  if (a.hist && p.root < a.hist_n)
    atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + 4ull * p.root), static_cast<unsigned long long>(q));
  p.ix = static_cast<int>(floorf((p.x - a.g.x0) * a.g.idx));
  p.iy = static_cast<int>(floorf((p.y - a.g.y0) * a.g.idy));
  p.iz = 0;
  if (p.ix < 0 || p.ix >= a.g.nx || p.iy < 0 || p.iy >= a.g.ny || p.w <= 0.0f) {
    escape(a, p, q, acc);
    return false;
  }
  return true;
}

// A primary as the phase-space kernel leaves it for the transport kernel: the state after
// spot sampling, ready to step.  Primaries start on the entrance face (iz = 0); ix < 0 marks
// one that was born outside the grid (its energy is already booked as escaped).
struct __align__(16) PrimaryRecord {
  float x, y, z, u;
  float v, w, E, nmfp;
  int ix, iy;
  unsigned root, b;
};
static_assert(sizeof(PrimaryRecord) == sizeof(Particle), "a primary record takes one queue slot");

__device__ __forceinline__ PrimaryRecord pack_primary(const PState& p, bool alive) {
  PrimaryRecord r;
  r.x = p.x; r.y = p.y; r.z = p.z; r.u = p.u; r.v = p.v; r.w = p.w; r.E = p.E; r.nmfp = p.nmfp;
  r.ix = alive ? p.ix : -1;
  r.iy = p.iy;
  r.root = p.root;
  r.b = p.b;
  return r;
}

// Takes a sampled primary; false for one born outside the grid.
__device__ __forceinline__ bool load_primary(const PrimaryRecord& r, PState& p) {
  p.x = r.x; p.y = r.y; p.z = r.z; p.u = r.u; p.v = r.v; p.w = r.w; p.E = r.E; p.nmfp = r.nmfp;
  p.ix = r.ix; p.iy = r.iy; p.iz = 0;
  p.root = r.root;
  p.pid = r.root;
  p.b = r.b;
  p.k = 0;
  p.fE = fix(p.E);
  return r.ix >= 0;
}

__device__ void init_queued(const TransportArgs& a, uint2 key, const Particle& r, PState& p) {
  p.x = r.x; p.y = r.y; p.z = r.z; p.u = r.u; p.v = r.v; p.w = r.w; p.E = r.E;
  p.pid = r.pid;
  p.root = r.root;
  p.b = r.root % static_cast<unsigned>(a.B);
  p.k = 0;
  p.fE = fix(p.E);
  p.nmfp = -logf(draw4(key, r.pid, 1u, 4u).x);
  const int nxy = a.g.nx * a.g.ny;
  p.iz = r.voxel / nxy;
  const int rem = r.voxel - p.iz * nxy;
  p.iy = rem / a.g.nx;
  p.ix = rem - p.iy * a.g.nx;
}

__device__ __forceinline__ Particle make_record(const PState& p, float E, float u, float v, float w,
                                                unsigned long long pid, int voxel, int target) {
  Particle r;
  r.x = p.x; r.y = p.y; r.z = p.z; r.u = u; r.v = v; r.w = w; r.E = E;
  r.voxel = voxel; r.pid = pid; r.root = p.root; r.target = target;
  return r;
}

// One condensed-history step (Sec. II.A.3).  Returns false when the particle ends.  kLet, kMol
// and kVav compile the LET scoring, the Moliere option and the Vavilov option in; without
// them the step carries no test for any of them.  The debug deposit log is a run-time switch
// (a.dlog) rather than a specialisation, so that a logged run executes the very instructions
// of an unlogged one: a separately compiled kernel may contract multiply-adds differently.
template <bool kLet, bool kMol, bool kVav, class Q>
__device__ bool step(const TransportArgs& a, const Physics& ph, const float2* rt, const float2* et,
                     const float* st, const float4* mol, uint2 key, PState& p, Acc& acc, Q& q) {
  const int v = vindex(a.g, p.ix, p.iy, p.iz);
  if (p.E <= kEcut) {
    const long long q = fix(p.E);
    deposit(a, v, p, q, acc);
    if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, 0.0, 0.0);
    if (kLet && p.E > 0.0f) {   // absorbed over its residual range: L = E / R
      int m0;
      float rho0;
      voxel_props(ph, a.g, v, m0, rho0);
      const MatConst& m0c = ph.mat[m0];
      const float R0 = range_mass(ph, rt, m0c.cls, p.E, logf(p.E)) / (rho0 * m0c.f);
      if (R0 > 0.0f) score_let(a, v, p, q, 0.1f * p.E / R0);
    }
    return false;
  }
  if (p.k >= kMaxSteps) {
    deposit(a, v, p, fix(p.E), acc);
    if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, 0.0, 0.0);
    acc.errors++;
    return false;
  }
  // the step's uniforms depend only on the particle's identity and step count: drawn
  // first, their Philox rounds interleave with the table lookups below
  const StepUniforms ua = step_uniforms(key, p.pid, p.k);
  int m;
  float rho;
  voxel_props(ph, a.g, v, m, rho);
  const MatConst& mc = ph.mat[m];
  const float E0 = p.E;
  const float lnE = logf(E0);
  const float Rm = range_mass(ph, rt, mc.cls, E0, lnE);
  const float rf = rho * mc.f;
  const float Rcm = Rm / rf;
  const float sig = sigma_table(ph, st, m, lnE) * rho;
  const float lam = sig > 0.0f ? p.nmfp / sig : 3.0e38f;
  int axis;
  const float d = voxel_exit(a.g, p.x, p.y, p.z, p.u, p.v, p.w, p.ix, p.iy, p.iz, axis);
  acc.steps++;
  if (Rcm <= lam && Rcm <= d) {
    const long long q = fix(E0);
    deposit(a, v, p, q, acc);
    if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, E0, 0.0, 0.0);
    if (kLet && Rcm > 0.0f) score_let(a, v, p, q, 0.1f * E0 / Rcm);
    return false;
  }
  bool nuclear = lam <= d;
  const float dx = nuclear ? lam : d;
  const float tau = ua.u4;
  const float x1 = p.x + tau * dx * p.u, y1 = p.y + tau * dx * p.v, z1 = p.z + tau * dx * p.w;
  if (kMol && !(ph.flags & kNoMcs)) {
    // Moliere (Bethe's form), at the step-start energy over the planned step
    const float pc = sqrtf(E0 * E0 + 2.0f * E0 * kMp);
    const float pb = pc * pc / (E0 + kMp);
    const float chic2 = mc.mol_K * dx * rho / (pb * pb);
    const float B = moliere_b(mol, m, lnE, dx * rho);
    const float th = moliere_theta(mol, ua.u0, chic2, B);
    if (th > 0.0f) {
      float s_, c_, sp, cp;
      sincosf(th, &s_, &c_);
      sincos_2pi(ua.u1, &sp, &cp);
      rotate(p.u, p.v, p.w, c_, s_, cp, sp);
    }
  } else if (!(ph.flags & kNoMcs)) {
    // Highland x 1.07 at the step-start energy, over the planned step: with e = E + M and
    // (pc)^2 = E (E + 2M), 1 / (beta p c) = e / (pc)^2 and x / (X0 beta^2) = (x / X0) e / (beta p c).
    // The two projected Gaussian angles th0 (r cos phi, r sin phi) deflect by th0 r at azimuth phi.
    const float e = E0 + kMp;
    const float pc2 = E0 * (E0 + 2.0f * kMp);
    const float xr = dx * rho * mc.inv_X0;
    if (xr > 0.0f) {
      const float ibpc = e / pc2;
      const float br = fmaxf(1.0f + 0.038f * logf(xr * e * ibpc), 0.0f);
      const float th = (1.07f * 13.6f) * ibpc * sqrtf(xr) * br * sqrtf(-2.0f * logf(ua.u0));
      if (th > 0.0f) {
        float sn, cs, s_, c_;
        sincos_2pi(ua.u1, &sn, &cs);
        sincosf(th, &s_, &c_);
        rotate(p.u, p.v, p.w, c_, s_, cs, sn);
      }
    }
  }
  float L2 = (1.0f - tau) * dx;
  int axis2;
  const float d2 = voxel_exit(a.g, x1, y1, z1, p.u, p.v, p.w, p.ix, p.iy, p.iz, axis2);
  bool crossing = false;
  if (d2 <= L2) { L2 = d2; crossing = true; nuclear = false; }
  const float s = tau * dx + L2;
  p.x = x1 + L2 * p.u; p.y = y1 + L2 * p.v; p.z = z1 + L2 * p.w;
  const float Rleft = Rm - s * rf;
  const float E_left = Rleft > 0.0f ? energy_of_range(ph, et, mc.cls, Rleft) : 0.0f;
  float dE = E0 - E_left;
  if (!(ph.flags & kNoStraggling)) {
    const float e = E0 + kMp;
    const float pc2 = E0 * (E0 + 2.0f * kMp);
    bool vav = false;
    if (kVav) {
      const float g = e * (1.0f / kMp);
      const float b2 = pc2 / (e * e);
      // Vavilov where kappa = xi / T_max <= 10: xi = (K/2)(Z/A) rho s / beta^2, T_max the
      // largest transfer to a free electron; beyond it Bohr's Gaussian (the same variance)
      const float r = kMe / kMp;
      const float tmax = 2.0f * kMe * b2 * g * g / (1.0f + 2.0f * g * r + r * r);
      const float xi = 0.5f * kKBethe * mc.ZA * rho * s / b2;
      const float kappa = xi / tmax;
      if (kappa <= 10.0f) {
        dE += xi * vavilov_z(a.vav, kappa, b2, ua.u2);
        vav = true;
      }
    }
    if (!vav) {
      // Bohr's variance with the relativistic factor (1 - beta^2/2) / (1 - beta^2) =
      // (e^2 - (pc)^2 / 2) / M^2
      const float var = mc.bohr_k * rho * s * (e * e - 0.5f * pc2) * (1.0f / (kMp * kMp));
      float sn, cs;
      sincos_2pi(ua.u3, &sn, &cs);
      dE += sqrtf(var * (-2.0f * logf(ua.u2))) * cs;
    }
  }
  dE = fminf(fmaxf(dE, 0.0f), E0);
  const float E1 = E0 - dE;
  {
    const long long f1 = fix(E1);
    const long long q = p.fE - f1;
    p.fE = f1;
    deposit(a, v, p, q, acc);
    if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, E0, E1, 0.0);
    if (kLet) {
      // mean stopping power over the path: the CSDA loss over s, taken as a difference
      // of two values of the inverse range table (free of the E -> R -> E round trip,
      // whose few-ulp error would dominate the loss over the short steps that end at
      // a voxel face)
      const float L = s > 0.0f ? 0.1f * (energy_of_range(ph, et, mc.cls, Rm) - E_left) / s : 0.0f;
      score_let(a, v, p, q, fmaxf(L, 0.0f));
    }
  }
  p.E = E1;
  p.nmfp -= sig * s;
  const unsigned kstep = p.k++;
  if (crossing) {
    const float dir = axis2 == 0 ? p.u : (axis2 == 1 ? p.v : p.w);
    const int inc = dir > 0.0f ? 1 : -1;
    int& idx = axis2 == 0 ? p.ix : (axis2 == 1 ? p.iy : p.iz);
    idx += inc;
    const int lim = axis2 == 0 ? a.g.nx : (axis2 == 1 ? a.g.ny : a.g.nz);
    if (idx < 0 || idx >= lim) {
      const long long q = fix(p.E);
      escape(a, p, q, acc);
      if (a.esc) {
        const unsigned long long i = atomicAdd(&a.cnt->esc_count, 1ull);
        if (i < a.esc_cap) {
          float* o = a.esc + 8 * i;
          o[0] = p.E; o[1] = p.x; o[2] = p.y; o[3] = p.z; o[4] = p.u; o[5] = p.v; o[6] = p.w;
          o[7] = static_cast<float>(p.root);
        }
      }
      return false;
    }
    return true;
  }
  if (!nuclear || p.E <= kEcut) return true;

  // Nuclear collision: channel and target from the step-start cross-sections
  const float4 ub = draw4(key, p.pid, kstep, 1u);
  float s_in = 0.0f, s_el = 0.0f;
  for (int j = 0; j < mc.n; ++j) {
    const NucConst& nc = ph.nuc[mc.nuc[j]];
    if (!(ph.flags & kNoInelastic)) s_in += mc.n_per_g[j] * sigma_inel(nc, E0);
    if (!(ph.flags & kNoElastic)) s_el += mc.n_per_g[j] * sigma_el(nc, E0);
  }
  const bool inel = ub.x * (s_in + s_el) < s_in;
  const float ut = ub.y * (inel ? s_in : s_el);
  int t = -1, last = 0;
  float cum = 0.0f;
  for (int j = 0; j < mc.n; ++j) {
    const NucConst& nc = ph.nuc[mc.nuc[j]];
    const float part = inel ? ((ph.flags & kNoInelastic) ? 0.0f : mc.n_per_g[j] * sigma_inel(nc, E0))
                            : ((ph.flags & kNoElastic) ? 0.0f : mc.n_per_g[j] * sigma_el(nc, E0));
    if (part > 0.0f) last = j;
    cum += part;
    if (ut < cum) { t = j; break; }
  }
  if (t < 0) t = last;   // ut at the rounded total: the last nucleus with a share
  const int nuc = mc.nuc[t];
  if (inel) {
    acc.inel++;
    if (!q.event(make_record(p, p.E, p.u, p.v, p.w, p.pid, v, nuc))) {
      acc.dropped++;
      deposit(a, v, p, fix(p.E), acc);
      if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, 0.0, 0.0);
    }
    return false;
  }
  acc.el++;
  const NucConst& nc = ph.nuc[nuc];
  const float4 ue = draw4(key, p.pid, kstep, 2u);
  const ElasticOut eo = elastic_kinematics(nc, p.E, ue.x, ue.y);
  float sp, cp;
  sincospif(2.0f * ue.z, &sp, &cp);
  const float u0 = p.u, v0 = p.v, w0 = p.w;
  rotate(p.u, p.v, p.w, eo.c1, sqrtf(fmaxf(0.0f, 1.0f - eo.c1 * eo.c1)), cp, sp);
  const long long qE = fix(p.E), q1 = fix(eo.T1);
  if (nc.A == 1 && eo.T2 > kEcut) {
    float ru = u0, rv = v0, rw = w0;
    rotate(ru, rv, rw, eo.c2, sqrtf(fmaxf(0.0f, 1.0f - eo.c2 * eo.c2)), -cp, -sp);
    const unsigned long long cid = child_pid(key, p.pid, 0x10000u + kstep);
    if (q.secondary(make_record(p, eo.T2, ru, rv, rw, cid, v, -1))) {
      acc.sec++;
      deposit(a, v, p, qE - q1 - fix(eo.T2), acc);   // rounding remainder only
      if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, eo.T1, eo.T2);
    } else {
      acc.dropped++;
      deposit(a, v, p, qE - q1, acc);
      if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, eo.T1, 0.0);
    }
  } else {
    deposit(a, v, p, qE - q1, acc);                  // recoil nucleus deposits locally
    if (a.dlog) log_deposit(a.dlog, a.dlog_count, a.dlog_cap, v, p.b, p.E, eo.T1, 0.0);
  }
  p.E = eo.T1;
  p.fE = q1;
  p.nmfp = -logf(ub.z);
  return true;
}


// Adds the lanes' counters to the run's (warp reduction, one atomic per warp and counter).
__device__ __forceinline__ void flush_transport_counters(const Acc& acc, Counters* c, bool primary) {
  auto wsum = [](unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  const unsigned long long inc = wsum(static_cast<unsigned long long>(acc.inc));
  const unsigned long long dep = wsum(static_cast<unsigned long long>(acc.dep));
  const unsigned long long esc = wsum(static_cast<unsigned long long>(acc.esc));
  const unsigned long long steps = wsum(acc.steps), el = wsum(acc.el), inel = wsum(acc.inel);
  const unsigned long long sec = wsum(acc.sec), dropped = wsum(acc.dropped), errors = wsum(acc.errors);
  if ((threadIdx.x & 31u) == 0) {
    if (inc) atomicAdd(&c->incident, inc);
    if (dep) atomicAdd(&c->deposited, dep);
    if (esc) atomicAdd(&c->escaped, esc);
    if (steps) atomicAdd(&c->steps, steps);
    if (steps && primary) atomicAdd(&c->steps_primary, steps);
    if (el) atomicAdd(&c->elastic, el);
    if (inel) atomicAdd(&c->inelastic, inel);
    if (sec) atomicAdd(&c->secondaries, sec);
    if (dropped) atomicAdd(&c->dropped, dropped);
    if (errors) atomicAdd(&c->errors, errors);
  }
}

// Queue policy of the generation kernel: events and recoil protons appended to global queues.
struct GlobalQueues {
  const TransportArgs& a;
  __device__ __forceinline__ bool event(const Particle& r) const { return push(a.qne, a.qne_count, a.qne_cap, r); }
  __device__ __forceinline__ bool secondary(const Particle& r) const {
    return push(a.qsec, a.qsec_count, a.qsec_cap, r);
  }
};

// Stages the physics block and the tables (ranges, inverse ranges, cross-sections and, for
// the Moliere option, its tables) in shared memory; returns the tables' addresses there.
struct StagedTables {
  const Physics* ph;
  const float2 *rt, *et;
  const float* st;
  const float4* mol;
  unsigned char* end;          // first byte after the tables (16-byte aligned)
};

template <bool kMol>
__device__ __forceinline__ StagedTables stage_transport_tables(const TransportArgs& a, unsigned char* smem) {
  Physics* php = reinterpret_cast<Physics*>(smem);
  {
    const int4* src = reinterpret_cast<const int4*>(a.phys);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(Physics) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int ncls = php->n_cls, nmat = php->n_mat;
  const size_t off_rt = (sizeof(Physics) + 15) / 16 * 16;
  float2* rt = reinterpret_cast<float2*>(smem + off_rt);
  float2* et = rt + ncls * kNE;
  float* st = reinterpret_cast<float*>(et + ncls * kNR);
  for (int i = threadIdx.x; i < ncls * kNE; i += blockDim.x) rt[i] = a.rtab[i];
  for (int i = threadIdx.x; i < ncls * kNR; i += blockDim.x) et[i] = a.etab[i];
  for (int i = threadIdx.x; i < nmat * kNS; i += blockDim.x) st[i] = a.stab[i];
  unsigned char* end = smem + ((reinterpret_cast<unsigned char*>(st + nmat * kNS) - smem) + 15) / 16 * 16;
  float4* mol = nullptr;
  if (kMol) {
    mol = reinterpret_cast<float4*>(end);
    const float4* src = a.mol;
    const int n4 = static_cast<int>(moliere_table_bytes(nmat) / sizeof(float4));
    for (int i = threadIdx.x; i < n4; i += blockDim.x) mol[i] = src[i];
    end += (moliere_table_bytes(nmat) + 15) / 16 * 16;
  }
  __syncthreads();
  return StagedTables{php, rt, et, st, mol, end};
}

}  // namespace
}  // namespace pmc
