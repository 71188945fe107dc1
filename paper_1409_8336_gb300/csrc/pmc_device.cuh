// pmc_device.cuh -- device data layout and single-precision physics routines
// of the GB300 proton transport engine.  Method: Wan Chan Tseung, Ma & Beltran,
// arXiv:1409.8336, Sec. II.A (physics) and II.B (GPU organisation).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pmc {

// ---------------------------------------------------------------------------
// constants (MeV, cm, g)
// ---------------------------------------------------------------------------
constexpr float kMp = 938.272088f;
constexpr float kMn = 939.565420f;
constexpr double kMpD = 938.272088;
constexpr double kMnD = 939.565420;
constexpr double kAmuD = 931.49410242;
constexpr float kEcut = 0.1f;                  // Sec. II.A.3
constexpr float kFix = 16777216.0f;            // tally unit 2^-24 MeV
constexpr double kFixD = 16777216.0;
constexpr float kCoulomb = 1.439964548f;       // e^2 / 4 pi eps0, MeV fm
constexpr float kMe = 0.51099895f;             // electron mass, MeV
constexpr float kKBethe = 0.307075f;           // 4 pi N_A r_e^2 m_e c^2, MeV cm^2 / mol
constexpr float kFm2PerMb = 0.1f;
// Tables are uniform in ln E or ln R with spacing 2^-6, so the table coordinate
// (ln x - origin) * 64 is computed without a rounded scale factor: a rounded
// 1/h would bias every step's energy loss the same way and drift the range.
constexpr float kTabScale = 64.0f;             // 1 / grid spacing
constexpr int kNE = 384;                       // range nodes: ln E in [0, 383/64], E in [1, 396] MeV
constexpr int kNR = 768;                       // inverse-range nodes per class: ln R from lnR0[cls]
constexpr int kNS = 544;                       // cross-section nodes: ln E from kLnS0
constexpr float kLnS0 = -2.3125f;              // floor(64 ln 0.1) / 64
constexpr int kMaxMat = 16, kMaxNuc = 16, kMaxNucPerMat = 12, kMaxHu = 16, kMaxCls = 4;
constexpr int kShells = 15;                    // Woods-Saxon shells, Sec. II.A.4
constexpr int kMaxZ = 24, kMaxA = 52;          // binding-energy table extent
constexpr int kBtabFloats = kMaxZ * kMaxA + kMaxA;   // binding energies, then A^(1/3)
constexpr int kIncStack = 32;                  // cascade particles per event
constexpr int kIncRetries = 1000;
constexpr int kIncCrossings = 1000;
constexpr int kIncIterations = 100000;          // flights per nucleon
constexpr int kEvapSteps = 64;
constexpr unsigned kMaxSteps = 100000u;        // per particle; exceeding it is an error
constexpr unsigned kNoStraggling = 1u, kNoMcs = 2u, kNoElastic = 4u, kNoInelastic = 8u, kMoliere = 16u,
                   kVavilov = 32u;
// Vavilov straggling table: quantiles of z = (loss - mean loss) / xi on kVavNB values of beta^2
// in [0, kVavB2Max], kVavNK values of ln kappa in [ln kVavK0, ln kVavK1] and kVavNU values of u
// in [kVavU0, 1 - kVavU0], each row shifted to mean zero (trilinear sampling keeps it).
constexpr int kVavNK = 41, kVavNB = 6, kVavNU = 513;
constexpr double kVavK0 = 0.001, kVavK1 = 10.0, kVavB2Max = 0.5, kVavU0 = 1e-4;
constexpr int kMolN = 1025;                    // Moliere distribution-function nodes on v in [0, kMolVmax]
constexpr float kMolVmax = 8.0f;
constexpr float kMolBmin = 4.5f;               // validity floor of the expansion (Bethe)
// B(b), the root of B - ln B = b, tabulated in the fourth component of the distribution
// table's nodes: node i at b = kMolB0 + i / kMolBScale (kMolB0 = 4.5 - ln 4.5, B = 4.5)
constexpr float kMolB0 = 2.99592471f;
constexpr float kMolBScale = 32.0f;
// A guide to the distribution table's inversion: for u in [k, k+1) / kMolGuide, node
// brackets [lo, hi] (16 bits each) with F(lo) <= u < F(hi) for every B >= 4.5.
constexpr int kMolGuide = 256;
// Device bytes of the Moliere tables: kMolN float4 nodes, the guide, then n_mat x kNS floats of G_m.
__host__ __device__ constexpr size_t moliere_table_bytes(int n_mat) {
  return kMolN * sizeof(float4) + kMolGuide * sizeof(unsigned) + static_cast<size_t>(n_mat) * kNS * sizeof(float);
}

// Learned stand-in of the event generator (quantile network).
constexpr int kSurrSlots = 4;                    // proton slots per event
constexpr int kSurrFeatures = 4 + 2 * kSurrSlots;   // E, slot, n_p, T[4], cos[4], local
constexpr int kSurrTargets = 6;                  // one-hot target slots
constexpr int kSurrIn = 32;                      // padded input width
constexpr int kSurrHidden = 256;
constexpr int kSurrOut = 16;                     // padded output width (10 used)
constexpr int kSurrLayers = 5;                   // 32-256-256-256-256-16
constexpr int kSurrTau = 10;                     // quantile levels per row

// ---------------------------------------------------------------------------
// device data
// ---------------------------------------------------------------------------
struct MatConst {
  float ZA;                        // Z/A of the mixture, mol/g
  float f;                         // Eq. 1 scaling factor (1 for own-table materials)
  float inv_X0;                    // 1 / X0, cm^2/g
  float bohr_k;                    // K m_e c^2 Z/A: Bohr variance per (rho x), MeV^2 cm^2/g
  int cls;                         // range-table class
  int n;
  int nuc[kMaxNucPerMat];
  float n_per_g[kMaxNucPerMat];    // atoms per gram x 1e-27 (so that n * sigma[mb] is cm^2/g)
  // Moliere: chi_c^2 = mol_K x / (p beta)^2 (x in g/cm^2); the rest of the B equation is
  // tabulated per material (moliere_b below)
  float mol_K;
};

struct NucConst {
  int Z, A;
  float a13;                       // A^(1/3)
  float bc;                        // Coulomb barrier of the non-elastic cross-section, MeV
  float sig_he;                    // high-energy limit of the non-elastic cross-section, mb
  float el;                        // elastic prefactor 12 mb A^(2/3)
  float mass;                      // nuclear mass, MeV
  int pad;
};

struct HuBin { int lo, hi, mat; float a, b; };

// Everything the kernels read besides the big tables; staged in shared memory.
struct alignas(16) Physics {
  int n_mat, n_nuc, n_hu, n_cls;
  unsigned flags;
  float S1[kMaxCls];               // mass stopping power at 1 MeV per class
  float R1[kMaxCls];               // mass range at 1 MeV per class
  float lnR0[kMaxCls];             // origin of the inverse table (a multiple of 2^-6)
  int nR[kMaxCls];                 // inverse-table nodes used per class
  MatConst mat[kMaxMat];
  NucConst nuc[kMaxNuc];
  HuBin hu[kMaxHu];
};

// Shell model of one target nucleus for the cascade (Sec. II.A.4).
struct NucleusModel {
  float r[kShells + 1];            // shell radii, fm
  float rho[2][kShells];           // [0] neutrons, [1] protons, fm^-3
  float pF[2][kShells];            // Fermi momentum, MeV/c
  float TF[2][kShells];            // Fermi kinetic energy, MeV
  float V[2][kShells];             // well depth = T_F + separation energy, MeV
  float Rout;
  int Z, A, pad;
};

// A queued particle: a secondary proton (Q_sec) or a non-elastic event (Q_ne).
struct __align__(16) Particle {
  float x, y, z, u;
  float v, w, E;
  int voxel;                       // linear voxel index
  unsigned long long pid;          // identity: keys its random numbers
  unsigned root;                   // primary history index (group = root % B)
  int target;                      // nuclide index (Q_ne only)
};
static_assert(sizeof(Particle) == 48, "particle record is 48 bytes");

// Run counters; energies in units of 2^-24 MeV (signed, two's complement).
struct Counters {
  unsigned long long incident, deposited, escaped, binding;
  unsigned long long steps, elastic, inelastic, secondaries, transparent, inc_retries;
  unsigned long long dropped, errors, esc_count, steps_primary;
  unsigned long long surrogate_events;   // events generated by the learned stand-in
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Uniform in (0,1) from the top 23 bits (exact in single precision).
__device__ __forceinline__ float u01(unsigned x) {
  return (static_cast<float>(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// Four uniforms of stream (pid, word2, tag).  Tags: 0, 1 step uniforms;
// 2 nuclear elastic; 3 cascade/evaporation draws; 4 birth; 5 child identity.
__device__ __forceinline__ float4 draw4(uint2 key, unsigned long long pid, unsigned w2, unsigned tag) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)pid, (unsigned)(pid >> 32), w2, tag), key);
  return make_float4(u01(r.x), u01(r.y), u01(r.z), u01(r.w));
}

__device__ __forceinline__ unsigned long long child_pid(uint2 key, unsigned long long pid, unsigned idx) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)pid, (unsigned)(pid >> 32), idx, 5u), key);
  return (unsigned long long)r.x | ((unsigned long long)r.y << 32);
}

// The five uniforms of step k: one Philox block (tag 0); four from the top 23
// bits of its words, the fifth from their unused low bits (9 + 9 + 5 bits).
struct StepUniforms { float u0, u1, u2, u3, u4; };
__device__ __forceinline__ StepUniforms step_uniforms(uint2 key, unsigned long long pid, unsigned k) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)pid, (unsigned)(pid >> 32), k, 0u), key);
  const unsigned low = ((r.x & 0x1FFu) << 14) | ((r.y & 0x1FFu) << 5) | (r.z & 0x1Fu);
  return {u01(r.x), u01(r.y), u01(r.z), u01(r.w), (static_cast<float>(low) + 0.5f) * (1.0f / 8388608.0f)};
}

// Fixed-point energy: deposits are differences of these, so a particle's
// deposits telescope exactly to its energy.  For e >= 0.5 MeV, e * 2^24 is the
// float's 24-bit significand shifted left (exact, integer unit only); below,
// it fits a 32-bit integer.
__device__ __forceinline__ long long fix(float e) {
  const unsigned b = __float_as_uint(e);
  const int ex = static_cast<int>((b >> 23) & 0xFFu);
  if (ex >= 126) return static_cast<long long>(static_cast<unsigned long long>((b & 0x7FFFFFu) | 0x800000u) << (ex - 126));
  return static_cast<long long>(__float2int_rn(e * kFix));
}
__device__ __forceinline__ long long fixd(double e) { return __double2ll_rn(e * kFixD); }

// ---------------------------------------------------------------------------
// tables (Sec. II.A.2): cubic splines stored as (y, M h^2 / 6) pairs
// ---------------------------------------------------------------------------
__device__ __forceinline__ float spline_eval(const float2* __restrict__ t, float s, int n) {
  int j = static_cast<int>(s);
  j = j < 0 ? 0 : (j > n - 2 ? n - 2 : j);
  const float t1 = s - static_cast<float>(j), t0 = 1.0f - t1;
  const float2 a = t[j], b = t[j + 1];
  return t0 * a.x + t1 * b.x + (t0 * t0 - 1.0f) * t0 * a.y + (t1 * t1 - 1.0f) * t1 * b.y;
}

// Mass CSDA range (g/cm^2) of a proton of energy E; lnE = log(E).
__device__ __forceinline__ float range_mass(const Physics& ph, const float2* __restrict__ rt, int cls, float E,
                                            float lnE) {
  if (E <= 1.0f) return 2.0f * sqrtf(E) / ph.S1[cls];
  return spline_eval(rt + cls * kNE, lnE * kTabScale, kNE);
}

// Inverse of range_mass.
__device__ __forceinline__ float energy_of_range(const Physics& ph, const float2* __restrict__ et, int cls, float R) {
  if (R <= 0.0f) return 0.0f;
  if (R <= ph.R1[cls]) {
    const float h = 0.5f * R * ph.S1[cls];
    return h * h;
  }
  return spline_eval(et + cls * kNR, (logf(R) - ph.lnR0[cls]) * kTabScale, ph.nR[cls]);
}

// Total macroscopic nuclear cross-section per unit density (cm^2/g), linear in ln E.
__device__ __forceinline__ float sigma_table(const Physics& ph, const float* __restrict__ st, int m, float lnE) {
  float s = (lnE - kLnS0) * kTabScale;
  s = fminf(fmaxf(s, 0.0f), static_cast<float>(kNS - 1) - 1e-3f);
  const int j = static_cast<int>(s);
  const float t = s - static_cast<float>(j);
  const float* p = st + m * kNS + j;
  return p[0] + t * (p[1] - p[0]);
}

// ---------------------------------------------------------------------------
// cross-sections (mb), the engine's analytic forms
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sigma_nn(float T, bool like) {
  const float t = fmaxf(T, 10.0f);
  const float g = 1.0f + t / kMp;
  const float b2 = 1.0f - 1.0f / (g * g);
  const float ib = rsqrtf(b2), ib2 = 1.0f / b2;
  return like ? (10.63f * ib2 - 29.92f * ib + 42.9f) : (34.10f * ib2 - 82.2f * ib + 82.2f);
}

// Non-elastic (Letaw, Silberberg & Tsao's fit to measured reaction cross-sections, closed
// below the Coulomb barrier).
__device__ __forceinline__ float sigma_inel(const NucConst& n, float E) {
  if (n.A <= 1 || E <= n.bc) return 0.0f;
  const float shape = 1.0f - 0.62f * expf(-E * (1.0f / 200.0f)) * sinf(10.9f * exp2f(-0.28f * log2f(E)));
  return n.sig_he * shape * (1.0f - n.bc / E);
}

__device__ __forceinline__ float sigma_el(const NucConst& n, float E) {
  if (E <= 0.0f) return 0.0f;
  if (n.A == 1) return sigma_nn(E, true);
  return n.el * (1.0f + 20.0f / (E + 10.0f));
}

// Moliere space angle for the uniform u (Bethe's form): the distribution function
// F0 + F1/B + F2/B^2 (nodes T[i] = (F0, F1, F2) at v = i h) inverted by bisection within
// the guide's bracket for u and linear interpolation; beyond kMolVmax the single-scattering tail
// (density ~ v^-3); theta = v chi_c sqrt(B), at most pi.
__device__ __forceinline__ float moliere_theta(const float4* T, float u, float chic2, float B) {
  const float iB = 1.0f / B, iB2 = iB * iB;
  auto F = [&](int i) {
    const float4 t = T[i];
    return t.x + t.y * iB + t.z * iB2;
  };
  const float Fmax = F(kMolN - 1);
  float v;
  if (u >= Fmax) {
    v = kMolVmax * sqrtf((1.0f - Fmax) / (1.0f - u));
  } else {
    const unsigned* guide = reinterpret_cast<const unsigned*>(T + kMolN);
    const unsigned gw = guide[min(static_cast<int>(u * static_cast<float>(kMolGuide)), kMolGuide - 1)];
    int lo = static_cast<int>(gw & 0xffffu), hi = static_cast<int>(gw >> 16);
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (F(mid) <= u) lo = mid; else hi = mid;
    }
    const float f0 = F(lo), f1 = F(hi);
    const float t = f1 > f0 ? (u - f0) / (f1 - f0) : 0.0f;
    v = (static_cast<float>(lo) + t) * (kMolVmax / static_cast<float>(kMolN - 1));
  }
  return fminf(v * sqrtf(chic2 * B), 3.14159265f);
}

// Moliere's B for a step of x = rho dx g/cm^2 of material m at ln E: b = ln chi_c^2 -
// ln(1.167 chi_a^2) = ln x + G_m(E), with G_m tabulated on the cross-section grid after the
// distribution table; B from the tabulated root of B - ln B = b (Newton beyond its end), and
// the expansion's floor 4.5 below b(4.5).
__device__ __forceinline__ float moliere_b(const float4* T, int m, float lnE, float x) {
  const float* G = reinterpret_cast<const float*>(T + kMolN) + kMolGuide;
  float s = (lnE - kLnS0) * kTabScale;
  s = fminf(fmaxf(s, 0.0f), static_cast<float>(kNS - 1) - 1e-3f);
  const int j = static_cast<int>(s);
  const float* g = G + m * kNS + j;
  const float b = logf(x) + (g[0] + (s - static_cast<float>(j)) * (g[1] - g[0]));
  if (!(b > kMolB0)) return kMolBmin;
  const float sb = (b - kMolB0) * kMolBScale;
  if (sb < static_cast<float>(kMolN - 1)) {
    const int i = static_cast<int>(sb);
    const float w0 = T[i].w, w1 = T[i + 1].w;
    return w0 + (sb - static_cast<float>(i)) * (w1 - w0);
  }
  float B = b + logf(b);
#pragma unroll
  for (int it = 0; it < 4; ++it) B -= (B - logf(B) - b) / (1.0f - 1.0f / B);
  return B;
}

// Vavilov straggling: the centred loss z (units of xi) for the uniform u at (kappa, beta^2),
// trilinear in (ln kappa, beta^2, u); kappa is clamped to the table's range.
__device__ __forceinline__ float vavilov_z(const float* __restrict__ T, float kappa, float b2, float u) {
  const float lk0 = static_cast<float>(-6.907755278982137), lk1 = static_cast<float>(2.302585092994046);
  const float a = (fminf(fmaxf(logf(kappa), lk0), lk1) - lk0) * ((kVavNK - 1) / (lk1 - lk0));
  const float b = fminf(fmaxf(b2, 0.0f), static_cast<float>(kVavB2Max)) * ((kVavNB - 1) / static_cast<float>(kVavB2Max));
  const float c = u * (kVavNU - 1);
  const int ia = min(static_cast<int>(a), kVavNK - 2), ib = min(static_cast<int>(b), kVavNB - 2);
  const int ic = min(static_cast<int>(c), kVavNU - 2);
  const float fa = a - ia, fb = b - ib, fc = c - ic;
  float v[2][2];
#pragma unroll
  for (int jb = 0; jb < 2; ++jb)
#pragma unroll
    for (int ja = 0; ja < 2; ++ja) {
      const float* row = T + (static_cast<size_t>(ib + jb) * kVavNK + (ia + ja)) * kVavNU + ic;
      v[jb][ja] = row[0] + fc * (row[1] - row[0]);
    }
  const float lo = v[0][0] + fa * (v[0][1] - v[0][0]), hi = v[1][0] + fa * (v[1][1] - v[1][0]);
  return lo + fb * (hi - lo);
}

// ---------------------------------------------------------------------------
// directions
// ---------------------------------------------------------------------------
// Rotates (u,v,w) to polar angle (ct, st) and azimuth (cp, sp) about itself.
__device__ __forceinline__ void rotate(float& u, float& v, float& w, float ct, float st, float cp, float sp) {
  const float s2 = 1.0f - w * w;
  float nu, nv, nw;
  if (s2 < 1e-10f) {
    nu = st * cp;
    nv = st * sp;
    nw = w >= 0.0f ? ct : -ct;
  } else {
    const float is = rsqrtf(s2), s = s2 * is;
    nu = u * ct + st * (u * w * cp - v * sp) * is;
    nv = v * ct + st * (v * w * cp + u * sp) * is;
    nw = w * ct - st * cp * s;
  }
  const float in = rsqrtf(nu * nu + nv * nv + nw * nw);
  u = nu * in;
  v = nv * in;
  w = nw * in;
}

// Vector (a0, a1, a2) given in the frame whose third axis is (u, v, w).
__device__ __forceinline__ float3 frame_to_lab(float u, float v, float w, float a0, float a1, float a2) {
  const float s2 = 1.0f - w * w;
  float3 o;
  if (s2 < 1e-10f) {
    o = make_float3(a0, a1, w >= 0.0f ? a2 : -a2);
  } else {
    const float is = rsqrtf(s2), s = s2 * is;
    o.x = a0 * u * w * is - a1 * v * is + a2 * u;
    o.y = a0 * v * w * is + a1 * u * is + a2 * v;
    o.z = -a0 * s + a2 * w;
  }
  const float in = rsqrtf(o.x * o.x + o.y * o.y + o.z * o.z);
  return make_float3(o.x * in, o.y * in, o.z * in);
}

// ---------------------------------------------------------------------------
// nuclear elastic kinematics (Sec. II.A.5, Eq. 3)
// ---------------------------------------------------------------------------
struct ElasticOut { float T1, c1, T2, c2, ccm; };

__device__ __forceinline__ ElasticOut elastic_kinematics(const NucConst& n, float E, float u0, float u1) {
  const float m = kMp, M = n.mass;
  const float plab = sqrtf(E * E + 2.0f * E * m), Elab = E + m;
  const float s = m * m + M * M + 2.0f * M * Elab;
  const float rs = sqrtf(s);
  const float pcm = plab * M / rs;
  float ct;
  if (n.A == 1) {
    ct = 2.0f * u1 - 1.0f;
  } else {
    const float A = static_cast<float>(n.A);
    float a1, b1, a2, b2;
    if (n.A <= 62) {
      a1 = powf(A, 1.63f); b1 = 14.5f * powf(A, 0.66f); a2 = 1.4f * powf(A, 0.33f); b2 = 10.0f;
    } else {
      a1 = powf(A, 1.33f); b1 = 60.0f * powf(A, 0.33f); a2 = 0.4f * powf(A, 0.4f); b2 = 10.0f;
    }
    const float p = pcm * 1e-3f, tmax = 4.0f * p * p;
    const float e1 = -expm1f(-b1 * tmax), e2 = -expm1f(-b2 * tmax);
    const float w1 = a1 * e1 / b1, w2 = a2 * e2 / b2;
    const bool first = u0 * (w1 + w2) < w1;
    const float b = first ? b1 : b2, eb = first ? e1 : e2;
    const float t = -log1pf(-u1 * eb) / b;
    ct = fminf(fmaxf(1.0f - t / (2.0f * p * p), -1.0f), 1.0f);
  }
  const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
  const float beta = plab / (Elab + M), gam = (Elab + M) / rs;
  const float e1 = sqrtf(pcm * pcm + m * m), e2 = sqrtf(pcm * pcm + M * M);
  const float p1z = gam * (pcm * ct + beta * e1), pt = pcm * st;
  const float p2z = gam * (-pcm * ct + beta * e2);
  // kinetic energy from the momentum (no cancellation against the rest mass)
  const float p1sq = p1z * p1z + pt * pt;
  float T1 = p1sq / (sqrtf(p1sq + m * m) + m);
  T1 = fminf(fmaxf(T1, 0.0f), E);
  ElasticOut o;
  o.T1 = T1;
  o.T2 = E - T1;
  o.c1 = p1z * rsqrtf(p1sq);
  const float n2 = p2z * p2z + pt * pt;
  o.c2 = n2 > 0.0f ? p2z * rsqrtf(n2) : 1.0f;
  o.ccm = ct;
  return o;
}

}  // namespace pmc
