// cascade_event.cuh -- the non-elastic event generator's physics (Sec. II.A.4): the
// intranuclear cascade as steps a driver strings together (attempt setup, one nucleon
// flight, the residual nucleus, emission of the cascade nucleons) and the evaporation chain,
// with the sink that routes an event's products (protons queued for transport, neutrons and
// leftover excitation escaping, fragments and the residual recoil deposited locally).
// Shared by the cascade kernels (cascade.cu) and the persistent drain kernel (drain.cu).
//
// Cascade: two-component Fermi gas in 15 constant-density shells of a Woods-Saxon profile;
// the incident proton enters at a random point of the projected disc and every nucleon is
// tracked between shell boundaries (refraction or reflection) and NN collisions (elastic,
// isotropic in the pair frame, Pauli-blocked below the local Fermi energy); the event is
// redrawn until at least one allowed collision occurred.  The excitation energy follows
// from energy and momentum conservation with the mass table.  Evaporation: Weisskopf-Ewing
// emission of n, p, d, t, He3 and alpha, isotropic in the rest frame.  Tracking is single
// precision; the energy and momentum bookkeeping and the evaporation kinematics are double
// precision so that the energy ledger closes to rounding.
#pragma once

#include "pmc_kernels.cuh"

namespace pmc {
namespace {

__device__ __constant__ int kEjZ[6] = {0, 1, 1, 1, 2, 2};
__device__ __constant__ int kEjA[6] = {1, 1, 2, 3, 3, 4};
__device__ __constant__ float kEjG[6] = {2.f, 2.f, 3.f, 2.f, 2.f, 1.f};

struct Stream {
  uint2 key;
  unsigned long long pid;
  unsigned draw;
  int pos;
  float4 buf;
  __device__ float next() {
    if (pos == 4) {
      buf = draw4(key, pid, draw++, 3u);
      pos = 0;
    }
    const float r = pos == 0 ? buf.x : (pos == 1 ? buf.y : (pos == 2 ? buf.z : buf.w));
    ++pos;
    return r;
  }
};

__device__ __forceinline__ float mom(float T, float m) { return sqrtf(T * T + 2.0f * T * m); }

__device__ __forceinline__ float binding(const float* bt, int Z, int A) {
  if (Z < 0 || A < 1 || Z > A || Z >= kMaxZ || A >= kMaxA) return 0.0f;
  return bt[Z * kMaxA + A];
}

// Width integral int_0^X (X - x) exp(2 sqrt(a x)) dx: closed form
// (exp(2Y)(Y^2 - 3Y/2 + 3/4) + Y^2/2 - 3/4)/a^2 with Y = sqrt(a X); below Y = 1,
// where the closed form cancels, its power series sum_{n>=4} c_n Y^n / a^2 with
// c_n = 2^(n-2)(n-1)(n-3)/n!, summed by Horner's rule to n = 18.
__device__ float width_integral(float X, float a) {
  if (X <= 0.0f) return 0.0f;
  const float Y = sqrtf(a * X);
  if (Y >= 1.0f) return (expf(2.0f * Y) * (Y * Y - 1.5f * Y + 0.75f) + 0.5f * Y * Y - 0.75f) / (a * a);
  constexpr float c[15] = {5.00000000e-01f, 5.33333333e-01f, 3.33333333e-01f, 1.52380952e-01f, 5.55555556e-02f,
                           1.69312169e-02f, 4.44444444e-03f, 1.02613436e-03f, 2.11640212e-04f, 3.94667061e-05f,
                           6.71873688e-06f, 1.05244550e-06f, 1.52698565e-07f, 2.06361862e-08f, 2.61023189e-09f};
  float h = c[14];
#pragma unroll
  for (int k = 13; k >= 0; --k) h = fmaf(h, Y, c[k]);
  const float Y2 = Y * Y;
  return h * Y2 * Y2 / (a * a);
}

// z in [0, X] with density z exp(2 sqrt(a (X - z))), exact rejection.
__device__ float evap_sample(Stream& st, float X, float a) {
  const float sq = sqrtf(a * X);
  for (int it = 0; it < 1000; ++it) {
    if (sq >= 1.0f) {
      const float T = sqrtf(X / a);
      const float u1 = st.next(), u2 = st.next(), u3 = st.next();
      const float z = -T * logf(u1 * u2);
      if (z > X) continue;
      if (u3 <= expf(2.0f * sqrtf(a * (X - z)) - 2.0f * sq + z / T)) return z;
    } else {
      const float u1 = st.next(), u2 = st.next();
      const float z = X * u1;
      if (u2 * X * expf(2.0f * sq) <= z * expf(2.0f * sqrtf(a * (X - z)))) return z;
    }
  }
  return 0.5f * X;
}

__device__ __forceinline__ float3 iso_dir(Stream& st) {
  const float c = 2.0f * st.next() - 1.0f;
  const float ph = st.next();
  float sn, cs;
  sincospif(2.0f * ph, &sn, &cs);
  const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
  return make_float3(s * cs, s * sn, c);
}

struct IncP {
  float rx, ry, rz, dx, dy, dz, T;
  int q, shell, done, refl;
};

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
  return ax * bx + ay * by + az * bz;
}

__device__ __forceinline__ float dist_out(const IncP& p, float R) {
  const float b = dot3(p.rx, p.ry, p.rz, p.dx, p.dy, p.dz);
  const float c = dot3(p.rx, p.ry, p.rz, p.rx, p.ry, p.rz) - R * R;
  const float disc = fmaxf(b * b - c, 0.0f);
  return fmaxf(-b + sqrtf(disc), 0.0f);
}

__device__ __forceinline__ float dist_in(const IncP& p, float R) {
  const float b = dot3(p.rx, p.ry, p.rz, p.dx, p.dy, p.dz);
  if (b >= 0.0f) return -1.0f;
  const float c = dot3(p.rx, p.ry, p.rz, p.rx, p.ry, p.rz) - R * R;
  const float disc = b * b - c;
  if (disc <= 0.0f) return -1.0f;
  return fmaxf(-b - sqrtf(disc), 0.0f);
}

// Refraction or reflection at a shell boundary; n is the unit normal into the
// region entered.  Returns true when the nucleon crossed.
__device__ bool cross_boundary(IncP& p, float nx, float ny, float nz, float Va, float Vb, float m) {
  const float Tb = p.T - Va + Vb;
  const float dn = dot3(p.dx, p.dy, p.dz, nx, ny, nz);
  if (Tb > 0.0f) {
    const float pa = mom(p.T, m), pb = mom(Tb, m);
    const float pt2 = pa * pa * (1.0f - dn * dn);
    const float pn2 = pb * pb - pt2;
    if (pn2 > 0.0f) {
      const float pn = sqrtf(pn2);
      float ux = (pa * (p.dx - dn * nx) + pn * nx) / pb;
      float uy = (pa * (p.dy - dn * ny) + pn * ny) / pb;
      float uz = (pa * (p.dz - dn * nz) + pn * nz) / pb;
      const float in = rsqrtf(ux * ux + uy * uy + uz * uz);
      p.dx = ux * in; p.dy = uy * in; p.dz = uz * in;
      p.T = Tb;
      return true;
    }
  }
  p.dx -= 2.0f * dn * nx; p.dy -= 2.0f * dn * ny; p.dz -= 2.0f * dn * nz;
  const float in = rsqrtf(p.dx * p.dx + p.dy * p.dy + p.dz * p.dz);
  p.dx *= in; p.dy *= in; p.dz *= in;
  return false;
}

// Isotropic elastic NN scattering in the pair frame (relativistic).
__device__ void nn_collide(float3 p1, float E1, float m1, float3 p2, float E2, float m2, float3 ns, float3& p1o,
                           float& T1o, float3& p2o, float& T2o) {
  const float Px = p1.x + p2.x, Py = p1.y + p2.y, Pz = p1.z + p2.z, Et = E1 + E2;
  const float s = Et * Et - (Px * Px + Py * Py + Pz * Pz);
  const float rs = sqrtf(s);
  const float k = sqrtf(fmaxf(0.0f, (s - (m1 + m2) * (m1 + m2)) * (s - (m1 - m2) * (m1 - m2)))) / (2.0f * rs);
  const float bx = Px / Et, by = Py / Et, bz = Pz / Et;
  const float b2 = bx * bx + by * by + bz * bz, gam = Et / rs;
  const float psx = k * ns.x, psy = k * ns.y, psz = k * ns.z;
  const float es = sqrtf(k * k + m1 * m1);
  const float bp = bx * psx + by * psy + bz * psz;
  const float coef = b2 > 0.0f ? ((gam - 1.0f) * bp / b2 + gam * es) : 0.0f;
  p1o = make_float3(psx + coef * bx, psy + coef * by, psz + coef * bz);
  p2o = make_float3(Px - p1o.x, Py - p1o.y, Pz - p1o.z);
  const float e1o = gam * (es + bp);
  T1o = e1o - m1;
  T2o = (Et - e1o) - m2;
}

// ---------------------------------------------------------------------------
// The event, as steps that a driver strings together: attempt setup, one flight
// of the current nucleon, the residual nucleus of a finished attempt, the
// emission of the cascade nucleons, and the evaporation chain.  A driver that
// calls them in order consumes the event's random stream exactly as a single
// sequential routine would, whatever it interleaves between events.
// ---------------------------------------------------------------------------
struct IncState {
  IncP p;                   // the nucleon in flight (P[ip] is stale while it flies)
  int ip, n, sea0, sea1, crossings, iters;
  bool any;
};

// Residual nucleus after a successful cascade attempt (double precision bookkeeping).
struct Residual {
  double Ex, px, py, pz, bind;
  int Z, A;
};

// Attempt setup: entry point uniform on the projected disc of the outer sphere,
// the incident proton refracted into the outer shell.
__device__ __forceinline__ void inc_setup(const NucleusModel& nu, float E, Stream& st, IncP* P, IncState& s) {
  s.n = 1;
  s.ip = 0;
  s.sea0 = nu.A - nu.Z;
  s.sea1 = nu.Z;
  s.any = false;
  s.crossings = 0;
  s.iters = 0;
  const float b = nu.Rout * sqrtf(st.next());
  float sph, cph;
  sincospif(2.0f * st.next(), &sph, &cph);
  IncP& p0 = s.p;
  p0.q = 1; p0.T = E; p0.done = 0; p0.refl = 0;
  p0.rx = b * cph; p0.ry = b * sph; p0.rz = -sqrtf(fmaxf(0.0f, nu.Rout * nu.Rout - b * b));
  p0.dx = 0.0f; p0.dy = 0.0f; p0.dz = 1.0f;
  const float ir = rsqrtf(p0.rx * p0.rx + p0.ry * p0.ry + p0.rz * p0.rz);
  cross_boundary(p0, -p0.rx * ir, -p0.ry * ir, -p0.rz * ir, 0.0f, nu.V[1][kShells - 1], kMp);
  p0.shell = kShells - 1;
}

// One flight of s.p: to the next shell boundary (refraction or reflection) or to
// a sampled NN collision (Pauli-blocked or not).  Returns true when the nucleon
// has finished (escaped: done = 1; captured or trapped: done = 2).
__device__ __forceinline__ bool inc_flight(const NucleusModel& nu, Stream& st, IncP* P, IncState& s) {
  IncP& p = s.p;
  const int q = p.q;
  const float m = q ? kMp : kMn;
  const int i = p.shell;
  if (p.T - nu.V[q][i] <= 0.0f) { p.done = 2; return true; }
  if (++s.iters > kIncIterations) { p.done = 2; return true; }   // bounded loop: captured
  const float s_out = dist_out(p, nu.r[i + 1]);
  const float s_in = i > 0 ? dist_in(p, nu.r[i]) : -1.0f;
  const bool inner = s_in >= 0.0f && s_in < s_out;
  const float s_b = inner ? s_in : s_out;
  const float sl = sigma_nn(p.T, true) * kFm2PerMb, su = sigma_nn(p.T, false) * kFm2PerMb;
  const float rate_p = s.sea1 > 0 ? nu.rho[1][i] * (q == 1 ? sl : su) : 0.0f;
  const float rate_n = s.sea0 > 0 ? nu.rho[0][i] * (q == 0 ? sl : su) : 0.0f;
  const float rate = rate_p + rate_n;
  const float uc = st.next();
  const float s_c = rate > 0.0f ? -logf(uc) / rate : 3.0e38f;
  if (s_c < s_b) {
    p.rx += s_c * p.dx; p.ry += s_c * p.dy; p.rz += s_c * p.dz;
    const int q2 = st.next() * rate < rate_p ? 1 : 0;
    const float m2 = q2 ? kMp : kMn;
    const float p2m = nu.pF[q2][i] * cbrtf(st.next());
    const float3 d2 = iso_dir(st);
    const float3 ns = iso_dir(st);
    const float p1m = mom(p.T, m);
    float3 p1o, p2o;
    float T1o, T2o;
    nn_collide(make_float3(p1m * p.dx, p1m * p.dy, p1m * p.dz), p.T + m, m,
               make_float3(p2m * d2.x, p2m * d2.y, p2m * d2.z), sqrtf(p2m * p2m + m2 * m2), m2, ns, p1o, T1o, p2o,
               T2o);
    if (T1o < nu.TF[q][i] || T2o < nu.TF[q2][i]) return false;   // Pauli blocked
    if (s.n >= kIncStack) return false;                           // stack full: treated as blocked
    const float i1 = rsqrtf(p1o.x * p1o.x + p1o.y * p1o.y + p1o.z * p1o.z);
    const float i2 = rsqrtf(p2o.x * p2o.x + p2o.y * p2o.y + p2o.z * p2o.z);
    p.dx = p1o.x * i1; p.dy = p1o.y * i1; p.dz = p1o.z * i1;
    p.T = T1o;
    p.refl = 0;
    IncP c;
    c.q = q2; c.T = T2o; c.shell = i; c.done = 0; c.refl = 0;
    c.rx = p.rx; c.ry = p.ry; c.rz = p.rz;
    c.dx = p2o.x * i2; c.dy = p2o.y * i2; c.dz = p2o.z * i2;
    P[s.n++] = c;
    if (q2 == 1) --s.sea1; else --s.sea0;
    s.any = true;
    return false;
  }
  p.rx += s_b * p.dx; p.ry += s_b * p.dy; p.rz += s_b * p.dz;
  if (++s.crossings > kIncCrossings) { p.done = 2; return true; }
  const float ir = rsqrtf(p.rx * p.rx + p.ry * p.ry + p.rz * p.rz);
  bool crossed;
  if (inner) {
    crossed = cross_boundary(p, -p.rx * ir, -p.ry * ir, -p.rz * ir, nu.V[q][i], nu.V[q][i - 1], m);
    if (crossed) p.shell = i - 1;
  } else {
    const float Vb = (i + 1 < kShells) ? nu.V[q][i + 1] : 0.0f;
    crossed = cross_boundary(p, p.rx * ir, p.ry * ir, p.rz * ir, nu.V[q][i], Vb, m);
    if (crossed) {
      if (i + 1 == kShells) { p.done = 1; return true; }
      p.shell = i + 1;
    }
  }
  if (!crossed && ++p.refl >= 2) { p.done = 2; return true; }
  return false;
}

// After the last nucleon of an attempt: the residual nucleus from energy and
// momentum conservation with the mass table.  False when the attempt must be
// redrawn (no allowed collision, an impossible residual, or E* < 0).
__device__ __forceinline__ bool inc_residual(const NucleusModel& nu, const float* bt, float E, const IncP* P,
                                             const IncState& s, Residual& r) {
  if (!s.any) return false;
  int zesc = 0, nesc = 0;
  double sumT = 0.0, prx = 0.0, pry = 0.0, prz = static_cast<double>(mom(E, kMp));
  for (int ip = 0; ip < s.n; ++ip) {
    if (P[ip].done != 1) continue;
    ++nesc;
    zesc += P[ip].q;
    sumT += static_cast<double>(P[ip].T);
    const double pm = static_cast<double>(mom(P[ip].T, P[ip].q ? kMp : kMn));
    prx -= pm * P[ip].dx; pry -= pm * P[ip].dy; prz -= pm * P[ip].dz;
  }
  const int Zr = nu.Z + 1 - zesc, Ar = nu.A + 1 - nesc;
  if (Ar < 1 || Zr < 0 || Zr > Ar) return false;
  const double dM = static_cast<double>(binding(bt, nu.Z, nu.A)) - static_cast<double>(binding(bt, Zr, Ar));
  const double Trec = (prx * prx + pry * pry + prz * prz) * static_cast<double>(0.5f / (Ar * static_cast<float>(kAmuD)));
  const double Ex = static_cast<double>(E) - sumT - Trec - dM;
  if (Ex < 0.0) return false;
  r.Ex = Ex; r.px = prx; r.py = pry; r.pz = prz; r.bind = dM; r.Z = Zr; r.A = Ar;
  return true;
}

// The cascade nucleons that escaped, as products 0..k-1; returns k.
template <class Sink>
__device__ __forceinline__ int inc_emit(const IncP* P, int n, Sink& sink) {
  int k = 0;
  for (int ip = 0; ip < n; ++ip) {
    if (P[ip].done != 1) continue;
    sink.product(k++, P[ip].q, static_cast<double>(P[ip].T), P[ip].dx, P[ip].dy, P[ip].dz);
  }
  return k;
}

// Evaporation chain of the residual (products k, k+1, ...), then the residual's
// recoil, leftover excitation and binding to the sink.
template <class Sink>
__device__ void evaporate(const float* bt, Stream& st, Residual r, int k, int retries, Sink& sink) {
  double Ex = r.Ex, bind = r.bind;
  int Zc = r.Z, Ac = r.A;
  double pcx = r.px, pcy = r.py, pcz = r.pz;
  for (int stp = 0; stp < kEvapSteps; ++stp) {
    float G[6], X[6], Vj[6];
    float Gs = 0.0f;
    const float Bc = binding(bt, Zc, Ac);
    const float Exf = static_cast<float>(Ex);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      G[j] = 0.0f;
      X[j] = 0.0f;
      Vj[j] = 0.0f;
      const int Zd = Zc - kEjZ[j], Ad = Ac - kEjA[j];
      if (Ad < 1 || Zd < 0 || Zd > Ad) continue;
      // widths in single precision; the chosen channel's energies are redone in double below
      const float Sf = Bc - binding(bt, Zd, Ad) - binding(bt, kEjZ[j], kEjA[j]);
      const float rsum = bt[kMaxZ * kMaxA + Ad] + bt[kMaxZ * kMaxA + kEjA[j]];
      Vj[j] = (kEjZ[j] > 0 && Zd > 0) ? kCoulomb * kEjZ[j] * Zd / (1.5f * rsum) : 0.0f;
      X[j] = Exf - Sf - Vj[j];
      if (X[j] <= 0.0f) continue;
      const float mu = static_cast<float>(kEjA[j] * Ad) / static_cast<float>(kEjA[j] + Ad);
      G[j] = kEjG[j] * mu * (1.5f * rsum) * (1.5f * rsum) * width_integral(X[j], Ad * 0.125f);
      Gs += G[j];
    }
    if (!(Gs > 0.0f)) break;
    const float uch = st.next() * Gs;
    float acc = 0.0f;
    int j = 5;
    for (int c = 0; c < 6; ++c) {
      acc += G[c];
      if (uch < acc) { j = c; break; }
    }
    while (G[j] <= 0.0f) --j;
    const int Zd = Zc - kEjZ[j], Ad = Ac - kEjA[j];
    const double Sj = static_cast<double>(Bc) - static_cast<double>(binding(bt, Zd, Ad)) -
                      static_cast<double>(binding(bt, kEjZ[j], kEjA[j]));
    const double Xd = Ex - Sj - static_cast<double>(Vj[j]);
    const float z = fminf(evap_sample(st, X[j], Ad * 0.125f), static_cast<float>(fmax(Xd, 0.0)));
    const double eps = static_cast<double>(Vj[j]) + z;
    const double Exd = Xd - z;
    const float aj = static_cast<float>(kEjA[j]);
    const float mu = aj * Ad / (aj + Ad) * static_cast<float>(kAmuD);
    const double ps = static_cast<double>(sqrtf(2.0f * mu * static_cast<float>(eps)));
    const float3 nd = iso_dir(st);
    // Galilean split with masses A u: the parent's velocity is shared
    const double vfac = static_cast<double>(1.0f / (Ac * static_cast<float>(kAmuD)));
    const double vx = pcx * vfac, vy = pcy * vfac, vz = pcz * vfac;
    const double mej = aj * kAmuD, md = Ad * kAmuD;
    const double ex = mej * vx + ps * nd.x, ey = mej * vy + ps * nd.y, ez = mej * vz + ps * nd.z;
    pcx = md * vx - ps * nd.x;
    pcy = md * vy - ps * nd.y;
    pcz = md * vz - ps * nd.z;
    const double pe2 = ex * ex + ey * ey + ez * ez;
    const float ipe = rsqrtf(static_cast<float>(pe2));
    sink.product(k++, j, pe2 * static_cast<double>(0.5f / (aj * static_cast<float>(kAmuD))),
                 static_cast<float>(ex) * ipe, static_cast<float>(ey) * ipe, static_cast<float>(ez) * ipe);
    bind += Sj;
    Zc = Zd;
    Ac = Ad;
    Ex = Exd;
  }
  const double Tres = (pcx * pcx + pcy * pcy + pcz * pcz) * static_cast<double>(0.5f / (Ac * static_cast<float>(kAmuD)));
  sink.residual(Zc, Ac, Tres, Ex, bind, retries);
}

// The whole event in one thread.  Sink receives products (index, species,
// kinetic energy, direction in the frame where the incident proton moves along
// +z), then the residual, or `transparent` when no attempt succeeded.
template <class Sink>
__device__ void nonelastic_event(const NucleusModel& nu, const float* bt, float E, uint2 key, unsigned long long pid,
                                 IncP* P, Sink& sink) {
  Stream st{key, pid, 0u, 4, make_float4(0.f, 0.f, 0.f, 0.f)};
  IncState s;
  int retries = 0;
  for (int attempt = 0; attempt < kIncRetries; ++attempt) {
    inc_setup(nu, E, st, P, s);
    for (;;) {
      if (!inc_flight(nu, st, P, s)) continue;
      P[s.ip] = s.p;
      if (++s.ip >= s.n) break;
      s.p = P[s.ip];
      s.crossings = 0;
      s.iters = 0;
    }
    Residual r;
    if (!inc_residual(nu, bt, E, P, s, r)) { ++retries; continue; }
    const int k = inc_emit(P, s.n, sink);
    evaporate(bt, st, r, k, retries, sink);
    return;
  }
  sink.transparent(retries);
}

// Sink of the transport path: products to the lab frame, protons queued.  Env supplies the
// tallies, the per-history ledger, the deposit log and where queued protons go.
template <class Env>
struct EventSink {
  Env env;
  uint2 key;
  Particle ev;
  unsigned b;
  long long dep, esc, bnd;
  unsigned long long sec, dropped, retries, n_transparent;
  // q = llrint(e 2^24): the deposit of energy e (MeV) at the event's voxel
  __device__ void add_dep(long long q, double e) {
    atomicAdd(env.tally() + static_cast<size_t>(ev.voxel) * env.B() + b, static_cast<unsigned long long>(q));
    if (env.dlog()) log_deposit(env.dlog(), env.dlog_count(), env.dlog_cap(), ev.voxel, b, e, 0.0, 0.0);
    dep += q;
    if (env.hist() && ev.root < env.hist_n())
      atomicAdd(reinterpret_cast<unsigned long long*>(env.hist() + 4ull * ev.root + 1), static_cast<unsigned long long>(q));
  }
  __device__ void add_esc(long long q) {
    esc += q;
    if (env.hist() && ev.root < env.hist_n())
      atomicAdd(reinterpret_cast<unsigned long long*>(env.hist() + 4ull * ev.root + 2), static_cast<unsigned long long>(q));
  }
  __device__ void add_bind(long long q) {
    bnd += q;
    if (env.hist() && ev.root < env.hist_n())
      atomicAdd(reinterpret_cast<unsigned long long*>(env.hist() + 4ull * ev.root + 3), static_cast<unsigned long long>(q));
  }
  __device__ void queue(float T, float3 d, unsigned idx) {
    Particle r;
    r.x = ev.x; r.y = ev.y; r.z = ev.z; r.u = d.x; r.v = d.y; r.w = d.z; r.E = T;
    r.voxel = ev.voxel; r.pid = child_pid(key, ev.pid, idx); r.root = ev.root; r.target = -1;
    if (env.push(r)) {
      ++sec;
    } else {
      ++dropped;
      add_dep(fix(T), T);
    }
  }
  __device__ void product(int k, int species, double T, float ax, float ay, float az) {
    if (species == 1) {
      const float Tf = static_cast<float>(T);
      if (Tf > kEcut) queue(Tf, frame_to_lab(ev.u, ev.v, ev.w, ax, ay, az), static_cast<unsigned>(k));
      else add_dep(fixd(T), T);
    } else if (species == 0) {
      add_esc(fixd(T));
    } else {
      add_dep(fixd(T), T);
    }
  }
  __device__ void residual(int, int, double Tres, double Ex, double bind, int r) {
    add_dep(fixd(Tres), Tres);
    add_esc(fixd(Ex));
    add_bind(fixd(bind));
    retries += r;
  }
  __device__ void transparent(int r) {
    retries += r;
    ++n_transparent;
    queue(ev.E, make_float3(ev.u, ev.v, ev.w), 0x20000u);
  }
};

// Environment of the cascade kernels: their argument block, protons to its secondary queue.
struct CascadeEnv {
  const CascadeArgs* a;
  __device__ __forceinline__ unsigned long long* tally() const { return a->tally; }
  __device__ __forceinline__ int B() const { return a->B; }
  __device__ __forceinline__ long long* hist() const { return a->hist; }
  __device__ __forceinline__ unsigned long long hist_n() const { return a->hist_n; }
  __device__ __forceinline__ DepositRecord* dlog() const { return a->dlog; }
  __device__ __forceinline__ unsigned long long* dlog_count() const { return a->dlog_count; }
  __device__ __forceinline__ unsigned long long dlog_cap() const { return a->dlog_cap; }
  __device__ __forceinline__ bool push(const Particle& r) const {
    const unsigned i = atomicAdd(a->qsec_count, 1u);
    if (i >= a->qsec_cap) return false;
    a->qsec[i] = r;
    return true;
  }
};
using TransportSink = EventSink<CascadeEnv>;

// Reduces a sink's counters over the warp and adds them to the run counters.
template <class Env>
__device__ __forceinline__ void flush_counters(const EventSink<Env>& sk, Counters* c) {
  auto wsum = [](unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  const unsigned long long dep = wsum(static_cast<unsigned long long>(sk.dep));
  const unsigned long long esc = wsum(static_cast<unsigned long long>(sk.esc));
  const unsigned long long bnd = wsum(static_cast<unsigned long long>(sk.bnd));
  const unsigned long long sec = wsum(sk.sec), dr = wsum(sk.dropped), rt = wsum(sk.retries), tr = wsum(sk.n_transparent);
  if ((threadIdx.x & 31u) == 0) {
    if (dep) atomicAdd(&c->deposited, dep);
    if (esc) atomicAdd(&c->escaped, esc);
    if (bnd) atomicAdd(&c->binding, bnd);
    if (sec) atomicAdd(&c->secondaries, sec);
    if (dr) atomicAdd(&c->dropped, dr);
    if (rt) atomicAdd(&c->inc_retries, rt);
    if (tr) atomicAdd(&c->transparent, tr);
  }
}

}  // namespace
}  // namespace pmc
