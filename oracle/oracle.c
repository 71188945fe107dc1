/*
 * oracle.c -- plain, slow FP64 CPU reference of the proton transport method of
 * Wan Chan Tseung, Ma & Beltran, "A fast GPU-based Monte Carlo simulation of
 * proton transport with detailed modeling of non-elastic interactions"
 * (arXiv:1409.8336).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; it is written from
 * the paper (and, where the paper is silent, from the stated readings listed
 * in the design notes) so that the two can be compared.
 *
 * Every quantity is double precision.  Histories are processed one at a time,
 * depth first (a history's secondaries are kept on a local stack); random
 * numbers are keyed by particle identity, so the processing order does not
 * change the result.
 *
 * Passages followed (paper sections / equations):
 *   Sec. II.A.1  voxel geometry, HU -> material and density
 *   Sec. II.A.2  stopping power scaling (Eq. 1), range scaling (Eq. 2),
 *                Highland multiple scattering x 1.07, energy straggling,
 *                local deposition of delta-ray energy
 *   Sec. II.A.3  step = min(lambda, d, R), random hinge, elastic/non-elastic
 *                choice by one uniform, termination rules, E_cut = 0.1 MeV
 *   Sec. II.A.4  target choice by relative non-elastic cross-sections,
 *                intranuclear cascade (two-component Fermi gas, Woods-Saxon
 *                density as 15 constant-density shells, Pauli blocking,
 *                refraction/reflection at shell boundaries, elastic NN only,
 *                retry until at least one Pauli-allowed collision),
 *                evaporation isotropic in the rest frame, secondary policy
 *   Sec. II.A.5  coherent nuclear elastic scattering, Ranft dsigma/dOmega (Eq. 3),
 *                relativistic two-body kinematics
 *   Sec. II.B.2  ten groups of N/10 protons for the statistical error
 *   Sec. II.A.2  (option) Moliere multiple scattering in Bethe's form instead of
 *                the Highland width
 *   Sec. IV      dose-averaged LET scored beside the dose (proton energy losses
 *                weighted by the mean stopping power of the local medium over
 *                the path of each loss; recoil nuclei and fragments excluded)
 *
 * Parity status: every routine here is pinned by the CPU tests (closed forms,
 * conservation laws, brute-force tallies, published reference values).
 */
#define _DEFAULT_SOURCE   /* j1() of the C library, used for the Moliere tables */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* physical constants (MeV, cm, g)                                     */
/* ------------------------------------------------------------------ */
static const double M_PROTON = 938.272088;
static const double M_NEUTRON = 939.565420;
static const double M_ELECTRON = 0.51099895;
static const double AMU = 931.49410242;
static const double K_BETHE = 0.307075;        /* 4 pi N_A r_e^2 m_e c^2, MeV cm^2/mol */
static const double FINE_STRUCTURE = 1.0 / 137.035999084;
static const double X0_CONST = 716.408;        /* A / (4 alpha r_e^2 N_A), g/cm^2 */
static const double N_AVOGADRO = 6.02214076e23;
static const double HBARC = 197.3269804;       /* MeV fm */
static const double COULOMB_E2 = 1.439964548;  /* e^2 / 4 pi eps0, MeV fm */
static const double E_CUT = 0.1;               /* Sec. II.A.3 */
static const double MB_TO_CM2 = 1e-27;
static const double FM2_PER_MB = 0.1;
static const double TWO_PI = 6.283185307179586476925286766559;
static const double PI = 3.14159265358979323846264338328;

#define OR_MAX_NUC_PER_MAT 12
#define OR_NO_STRAGGLING 1u
#define OR_NO_MCS 2u
#define OR_NO_ELASTIC 4u
#define OR_NO_INELASTIC 8u
#define OR_MOLIERE 16u   /* Moliere multiple scattering instead of Highland */
#define OR_VAVILOV 32u   /* Vavilov straggling (table set by or_set_vavilov) where kappa <= 10 */

/* ------------------------------------------------------------------ */
/* public structures (mirrored by oracle.py with ctypes)               */
/* ------------------------------------------------------------------ */
typedef struct { int Z, A; double mass_u, I_eV; } or_nuclide;
typedef struct {
    int n; int nuc[OR_MAX_NUC_PER_MAT]; double w[OR_MAX_NUC_PER_MAT];
    double rho; double I_eV; int own_table;
} or_material;
typedef struct { int lo, hi, material; double rho_a, rho_b; } or_hu_bin;
typedef struct { double E, sigma_E, x, y, sigma_x, sigma_y, u, v, w, weight; } or_spot;
typedef struct {
    int n_nuc; const or_nuclide* nuc;
    int n_mat; const or_material* mat;
    int n_hu; const or_hu_bin* hu;
    int nx, ny, nz; double dx, dy, dz, x0, y0, z0;
    const int16_t* hu_vol; const uint8_t* mat_vol; const float* rho_vol;
    int n_spots; const or_spot* spots;
    int n_batches; unsigned flags;
} or_problem;

typedef struct {
    double incident, deposited, escaped, binding;
    double steps, elastic, inelastic, secondaries, transparent, inc_retries, errors;
} or_totals;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), own implementation */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Uniform in (0,1): the top 23 bits of a word, offset by half a step (a value
 * that single precision also represents exactly). */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Four uniforms of stream (pid, word2, tag) under key = seed. */
static void draw4(uint64_t seed, uint64_t pid, uint32_t word2, uint32_t tag, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), word2, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = u01(r[i]);
}

/* The five uniforms of step k of particle pid: one Philox block (tag 0); four
 * from the top 23 bits of its words, the fifth from their unused low bits
 * (9 + 9 + 5 bits of words 0, 1, 2). */
static void step_uniforms(uint64_t seed, uint64_t pid, uint32_t k, double u[5])
{
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), k, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = u01(r[i]);
    uint32_t low = ((r[0] & 0x1FFu) << 14) | ((r[1] & 0x1FFu) << 5) | (r[2] & 0x1Fu);
    u[4] = ((double)low + 0.5) * (1.0 / 8388608.0);
}

/* Identity of the child with index `idx` of particle `pid`. */
static uint64_t child_pid(uint64_t seed, uint64_t pid, uint32_t idx)
{
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), idx, 5u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    return (uint64_t)r[0] | ((uint64_t)r[1] << 32);
}

/* Sequential uniform stream used by one nuclear event (tag 3). */
typedef struct { uint64_t seed, pid; uint32_t draw; int pos; double buf[4]; } or_stream;
static double next_u(or_stream* s)
{
    if (s->pos == 4) { draw4(s->seed, s->pid, s->draw++, 3u, s->buf); s->pos = 0; }
    return s->buf[s->pos++];
}

/* ------------------------------------------------------------------ */
/* nuclear masses: Weizsaecker formula, measured light-nucleus binding */
/* ------------------------------------------------------------------ */
double or_binding_energy(int Z, int A)
{
    int N = A - Z;
    if (A <= 1 || Z < 0 || N < 0) return 0.0;
    if (A == 2) return (Z == 1) ? 2.224566 : 0.0;
    if (A == 3) return (Z == 1) ? 8.481798 : (Z == 2 ? 7.718043 : 0.0);
    if (A == 4) return (Z == 2) ? 28.295660 : 0.0;
    double a = (double)A, z = (double)Z;
    double b = 15.75 * a - 17.8 * pow(a, 2.0 / 3.0) - 0.711 * z * (z - 1.0) / cbrt(a)
             - 23.7 * (a - 2.0 * z) * (a - 2.0 * z) / a;
    if ((Z % 2 == 0) && (N % 2 == 0)) b += 11.18 / sqrt(a);
    else if ((Z % 2 == 1) && (N % 2 == 1)) b -= 11.18 / sqrt(a);
    return b > 0.0 ? b : 0.0;
}
double or_nuclear_mass(int Z, int A)
{
    return Z * M_PROTON + (A - Z) * M_NEUTRON - or_binding_energy(Z, A);
}

/* ------------------------------------------------------------------ */
/* stopping power, range, radiation length (Sec. II.A.2)               */
/* ------------------------------------------------------------------ */
/* Bethe mass stopping power, no shell or density correction; below 1 MeV it
 * is continued as S(1 MeV) * sqrt(E / 1 MeV). */
static double bethe_raw(double E, double ZA, double I_MeV)
{
    double g = 1.0 + E / M_PROTON;
    double b2 = 1.0 - 1.0 / (g * g);
    double bg2 = b2 * g * g;
    double r = M_ELECTRON / M_PROTON;
    double tmax = 2.0 * M_ELECTRON * bg2 / (1.0 + 2.0 * g * r + r * r);
    return K_BETHE * ZA / b2 * (0.5 * log(2.0 * M_ELECTRON * bg2 * tmax / (I_MeV * I_MeV)) - b2);
}
double or_mass_stopping_power(double E, double ZA, double I_eV)
{
    double I = I_eV * 1e-6;
    if (E >= 1.0) return bethe_raw(E, ZA, I);
    return bethe_raw(1.0, ZA, I) * sqrt(E);
}

/* Range table of one stopping-power class: R(E) is the integral of 1/S from
 * 0 to E.  Below 1 MeV it is 2 sqrt(E)/S(1); above, node values come from
 * 10-point Gauss-Legendre per interval and the interpolant is the cubic
 * Hermite polynomial with the exact slopes 1/S at the nodes. */
#define OR_RNODES 4001
typedef struct { double ZA, I_eV, S1, lnE0, dlnE; double E[OR_RNODES], R[OR_RNODES], dR[OR_RNODES]; } or_range_table;

static const double GL10_X[5] = {0.1488743389816312, 0.4333953941292472, 0.6794095682990244,
                                 0.8650633666889845, 0.9739065285171717};
static const double GL10_W[5] = {0.2955242247147529, 0.2692667193099963, 0.2190863625159820,
                                 0.1494513491505806, 0.0666713443086881};

static void range_table_build(or_range_table* t, double ZA, double I_eV)
{
    t->ZA = ZA; t->I_eV = I_eV;
    t->S1 = or_mass_stopping_power(1.0, ZA, I_eV);
    t->lnE0 = 0.0;
    t->dlnE = log(400.0) / (OR_RNODES - 1);
    for (int j = 0; j < OR_RNODES; ++j) t->E[j] = exp(t->lnE0 + j * t->dlnE);
    t->E[0] = 1.0;
    t->R[0] = 2.0 / t->S1;
    for (int j = 0; j < OR_RNODES; ++j) t->dR[j] = 1.0 / or_mass_stopping_power(t->E[j], ZA, I_eV);
    for (int j = 1; j < OR_RNODES; ++j) {
        double a = t->E[j - 1], b = t->E[j], m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
        for (int k = 0; k < 5; ++k)
            s += GL10_W[k] * (1.0 / or_mass_stopping_power(m - h * GL10_X[k], ZA, I_eV)
                            + 1.0 / or_mass_stopping_power(m + h * GL10_X[k], ZA, I_eV));
        t->R[j] = t->R[j - 1] + h * s;
    }
}

static double hermite(double x0, double x1, double y0, double y1, double d0, double d1, double x)
{
    double h = x1 - x0, t = (x - x0) / h, t2 = t * t, t3 = t2 * t;
    return (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * h * d0 + (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * h * d1;
}

static double range_of_energy(const or_range_table* t, double E)
{
    if (E <= 0.0) return 0.0;
    if (E <= 1.0) return 2.0 * sqrt(E) / t->S1;
    int j = (int)floor((log(E) - t->lnE0) / t->dlnE);
    if (j < 0) j = 0;
    if (j > OR_RNODES - 2) j = OR_RNODES - 2;
    while (j > 0 && t->E[j] > E) --j;
    while (j < OR_RNODES - 2 && t->E[j + 1] < E) ++j;
    return hermite(t->E[j], t->E[j + 1], t->R[j], t->R[j + 1], t->dR[j], t->dR[j + 1], E);
}

/* Inverse of range_of_energy, by bisection on the node table and then on
 * the monotone interpolant (to machine precision). */
static double energy_of_range(const or_range_table* t, double R)
{
    if (R <= 0.0) return 0.0;
    if (R <= t->R[0]) { double s = 0.5 * R * t->S1; return s * s; }
    int lo = 0, hi = OR_RNODES - 1;
    if (R >= t->R[hi]) return t->E[hi];
    while (hi - lo > 1) { int mid = (lo + hi) / 2; if (t->R[mid] <= R) lo = mid; else hi = mid; }
    double a = t->E[lo], b = t->E[lo + 1];
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b);
        if (m <= a || m >= b) break;
        double r = hermite(t->E[lo], t->E[lo + 1], t->R[lo], t->R[lo + 1], t->dR[lo], t->dR[lo + 1], m);
        if (r < R) a = m; else b = m;
    }
    return 0.5 * (a + b);
}

/* Tsai radiation length of one element (g/cm^2). */
double or_radiation_length_element(int Z, double A)
{
    double Lrad, Lp;
    switch (Z) {
    case 1: Lrad = 5.31; Lp = 6.144; break;
    case 2: Lrad = 4.79; Lp = 5.621; break;
    case 3: Lrad = 4.74; Lp = 5.805; break;
    case 4: Lrad = 4.71; Lp = 5.924; break;
    default: Lrad = log(184.15 / cbrt((double)Z)); Lp = log(1194.0 / pow((double)Z, 2.0 / 3.0));
    }
    double a2 = (FINE_STRUCTURE * Z) * (FINE_STRUCTURE * Z);
    double f = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
    return X0_CONST * A / ((double)Z * Z * (Lrad - f) + (double)Z * Lp);
}

/* Highland projected-angle width x 1.07 (Sec. II.A.2), path x, X0 in cm. */
double or_highland_theta0(double E, double x, double X0cm)
{
    if (x <= 0.0) return 0.0;
    double pc = sqrt(E * E + 2.0 * E * M_PROTON);
    double beta = pc / (E + M_PROTON);
    double br = 1.0 + 0.038 * log(x / (X0cm * beta * beta));
    if (br < 0.0) br = 0.0;
    return 1.07 * 13.6 / (beta * pc) * sqrt(x / X0cm) * br;
}

/* ------------------------------------------------------------------ */
/* Moliere multiple scattering, in Bethe's (1953) form: an option beside  */
/* the paper's Highland width (Sec. II.A.2).                              */
/* ------------------------------------------------------------------ */
/* The space angle theta = v chi_c sqrt(B) has the density
 *   [f0(v) + f1(v)/B + f2(v)/B^2] v dv,  f0 = 2 exp(-v^2),
 *   f_n(v) = (1/n!) int_0^inf u J0(v u) exp(-u^2/4) [(u^2/4) ln(u^2/4)]^n du,
 * so its distribution function is F0 + F1/B + F2/B^2 with F0 = 1 - exp(-v^2) and,
 * since int_0^v J0(t u) t dt = v J1(v u)/u,
 *   F_n(v) = (1/n!) int_0^inf v J1(v u) exp(-u^2/4) [(u^2/4) ln(u^2/4)]^n du.
 * F1 and F2 are tabulated by Simpson's rule on [0, MOL_VMAX]; beyond it the density is
 * read as its single-scattering tail, proportional to v^-3.  B solves
 * B - ln B = ln(chi_c^2 / (1.167 chi_a^2)); the expansion needs B >= 4.5 (Bethe), so
 * thinner steps take B = 4.5. */
#define MOL_N 1601
#define MOL_VMAX 8.0
#define MOL_BMIN 4.5
static double mol_F1[MOL_N], mol_F2[MOL_N];
static int mol_ready = 0;

static void mol_build(void)
{
    const int NU = 4000;
    const double U = 14.0, h = U / NU;
    for (int i = 0; i < MOL_N; ++i) {
        double v = MOL_VMAX * i / (MOL_N - 1), s1 = 0.0, s2 = 0.0;
        for (int k = 1; k <= NU; ++k) {         /* the integrand vanishes at u = 0 */
            double u = k * h, y = 0.25 * u * u, L = y * log(y);
            double g = v * j1(v * u) * exp(-y);
            double wk = (k == NU) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
            s1 += wk * g * L;
            s2 += wk * g * L * L;
        }
        mol_F1[i] = s1 * h / 3.0;
        mol_F2[i] = 0.5 * s2 * h / 3.0;
    }
    mol_ready = 1;
}

/* F_n(v) for n = 0, 1, 2 (linear interpolation of the tables for n > 0) */
double or_moliere_F(double v, int n)
{
    if (!mol_ready) mol_build();
    if (n == 0) return 1.0 - exp(-v * v);
    double x = v / MOL_VMAX * (MOL_N - 1);
    if (x < 0.0) x = 0.0;
    int i = (int)x;
    if (i > MOL_N - 2) i = MOL_N - 2;
    double t = x - i;
    if (t > 1.0) t = 1.0;
    const double* F = n == 1 ? mol_F1 : mol_F2;
    return F[i] + t * (F[i + 1] - F[i]);
}

static double mol_cdf(double v, double B)
{
    return or_moliere_F(v, 0) + or_moliere_F(v, 1) / B + or_moliere_F(v, 2) / (B * B);
}

/* chi_c^2 (rad^2) and B for a proton of kinetic energy E over mass thickness x
 * (g/cm^2) of material m */
void or_moliere_params(const or_problem* P, int m, double E, double x, double* chic2, double* B)
{
    const or_material* M = &P->mat[m];
    double pc = sqrt(E * E + 2.0 * E * M_PROTON), beta = pc / (E + M_PROTON);
    double zz = 0.0, lna = 0.0;
    for (int k = 0; k < M->n; ++k) {
        const or_nuclide* nu = &P->nuc[M->nuc[k]];
        double Z = nu->Z, c = M->w[k] * Z * (Z + 1.0) / nu->mass_u;
        double chi0 = 197.3269804 / (0.885 * 52917.721090) * cbrt(Z) / pc;   /* hbar c/(0.885 a0) Z^1/3 / pc */
        double alpha = Z / (137.035999 * beta);
        zz += c;
        lna += c * log(chi0 * chi0 * (1.13 + 3.76 * alpha * alpha));
    }
    lna /= zz;
    *chic2 = K_BETHE * M_ELECTRON * x * zz / (pc * beta * pc * beta);
    double b = log(*chic2) - lna - (2.0 * 0.5772156649015329 - 1.0);
    double Bv = MOL_BMIN;
    if (b > MOL_BMIN - log(MOL_BMIN)) {
        Bv = b + log(b);
        for (int it = 0; it < 100; ++it) {
            double d = (Bv - log(Bv) - b) / (1.0 - 1.0 / Bv);
            Bv -= d;
            if (fabs(d) < 1e-13 * Bv) break;
        }
        if (Bv < MOL_BMIN) Bv = MOL_BMIN;
    }
    *B = Bv;
}

/* The space angle for the uniform u: the distribution function inverted by bisection,
 * the tail beyond MOL_VMAX as v^-3, theta capped at pi. */
double or_moliere_theta(double u, double chic2, double B)
{
    double Fmax = mol_cdf(MOL_VMAX, B), v;
    if (u >= Fmax) {
        v = MOL_VMAX * sqrt((1.0 - Fmax) / (1.0 - u));
    } else {
        double lo = 0.0, hi = MOL_VMAX;
        for (int it = 0; it < 80; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mol_cdf(mid, B) < u) lo = mid; else hi = mid;
        }
        v = 0.5 * (lo + hi);
    }
    double th = v * sqrt(chic2 * B);
    return th < 0.5 * TWO_PI ? th : 0.5 * TWO_PI;
}

/* Vavilov straggling (optional; the paper uses Bohr's Gaussian).  The table, built by the
 * oracle's Python side from the characteristic function of the Bethe collision spectrum
 * (oracle/vavilov.py), holds quantiles of z = (loss - mean loss) / xi on OR_VAV_NB values of
 * beta^2 in [0, 0.5], OR_VAV_NK values of ln kappa in [ln 0.001, ln 10] and OR_VAV_NU values of
 * u in [1e-4, 1 - 1e-4], each row shifted to mean zero; sampled by trilinear interpolation. */
#define OR_VAV_NK 41
#define OR_VAV_NB 6
#define OR_VAV_NU 513
static double or_vav_tab[OR_VAV_NB * OR_VAV_NK * OR_VAV_NU];
static int or_vav_ready = 0;

void or_set_vavilov(const double* tab)
{
    memcpy(or_vav_tab, tab, sizeof(or_vav_tab));
    or_vav_ready = 1;
}

/* xi = (K/2)(Z/A) rho x / beta^2 (MeV) and kappa = xi / T_max of a proton of energy E over x cm. */
void or_vavilov_params(double E, double rho, double ZA, double x, double* xi, double* kappa)
{
    double g = 1.0 + E / M_PROTON;
    double b2 = 1.0 - 1.0 / (g * g);
    double r = M_ELECTRON / M_PROTON;
    double tmax = 2.0 * M_ELECTRON * b2 * g * g / (1.0 + 2.0 * g * r + r * r);
    *xi = 0.5 * K_BETHE * ZA * rho * x / b2;
    *kappa = *xi / tmax;
}

double or_vavilov_z(double kappa, double b2, double u)
{
    double lk = log(kappa < 0.001 ? 0.001 : (kappa > 10.0 ? 10.0 : kappa));
    double a = (lk - log(0.001)) / (log(10.0) - log(0.001)) * (OR_VAV_NK - 1);
    double b = (b2 < 0.0 ? 0.0 : (b2 > 0.5 ? 0.5 : b2)) / 0.5 * (OR_VAV_NB - 1);
    double cc = u * (OR_VAV_NU - 1);
    int ia = (int)a, ib = (int)b, ic = (int)cc;
    if (ia > OR_VAV_NK - 2) ia = OR_VAV_NK - 2;
    if (ib > OR_VAV_NB - 2) ib = OR_VAV_NB - 2;
    if (ic > OR_VAV_NU - 2) ic = OR_VAV_NU - 2;
    double fa = a - ia, fb = b - ib, fc = cc - ic;
    double v[2][2];
    for (int jb = 0; jb < 2; ++jb)
        for (int ja = 0; ja < 2; ++ja) {
            const double* row = or_vav_tab + ((size_t)(ib + jb) * OR_VAV_NK + (ia + ja)) * OR_VAV_NU;
            v[jb][ja] = row[ic] + fc * (row[ic + 1] - row[ic]);
        }
    double lo = v[0][0] + fa * (v[0][1] - v[0][0]);
    double hi = v[1][0] + fa * (v[1][1] - v[1][0]);
    return lo + fb * (hi - lo);
}

/* Bohr energy-loss straggling variance (MeV^2) over path x (cm). */
double or_bohr_variance(double E, double rho, double ZA, double x)
{
    double g = 1.0 + E / M_PROTON;
    double b2 = 1.0 - 1.0 / (g * g);
    return K_BETHE * M_ELECTRON * rho * ZA * x * (1.0 - 0.5 * b2) / (1.0 - b2);
}

/* ------------------------------------------------------------------ */
/* cross-sections (mb)                                                 */
/* ------------------------------------------------------------------ */
/* Free nucleon-nucleon elastic cross-sections, smooth fit in the lab
 * velocity of the projectile; energies below 10 MeV are evaluated at 10 MeV. */
double or_sigma_nn(double T, int like)
{
    double t = T < 10.0 ? 10.0 : T;
    double g = 1.0 + t / M_PROTON;
    double b = sqrt(1.0 - 1.0 / (g * g));
    if (like) return 10.63 / (b * b) - 29.92 / b + 42.9;
    return 34.10 / (b * b) - 82.2 / b + 82.2;
}

/* Proton-nucleus non-elastic cross-section.  The paper tabulates Geant4's values (Sec.
 * II.A.4), which are not available here; the reading is the empirical fit of Letaw,
 * Silberberg & Tsao (Astrophys. J. Suppl. 51 (1983) 271) to measured proton reaction
 * cross-sections,
 *   sigma_HE = 45 A^0.7 [1 + 0.016 sin(5.3 - 2.63 ln A)] mb,
 *   sigma(E) = sigma_HE [1 - 0.62 exp(-E/200) sin(10.9 E^-0.28)]   (E in MeV),
 * closed below the Coulomb barrier B_c = e^2 Z / (1.16 (A^1/3 + 1) fm) by the factor
 * (1 - B_c/E). */
double or_sigma_inelastic(int Z, int A, double E)
{
    if (A <= 1 || E <= 0.0) return 0.0;
    double a13 = cbrt((double)A);
    double bc = COULOMB_E2 * Z / (1.16 * (a13 + 1.0));
    if (E <= bc) return 0.0;
    double s_he = 45.0 * pow((double)A, 0.7) * (1.0 + 0.016 * sin(5.3 - 2.63 * log((double)A)));
    double shape = 1.0 - 0.62 * exp(-E / 200.0) * sin(10.9 * pow(E, -0.28));
    return s_he * shape * (1.0 - bc / E);
}

double or_sigma_elastic(int Z, int A, double E)
{
    (void)Z;
    if (E <= 0.0) return 0.0;
    if (A == 1) return or_sigma_nn(E, 1);
    return 12.0 * pow((double)A, 2.0 / 3.0) * (1.0 + 20.0 / (E + 10.0));
}

/* ------------------------------------------------------------------ */
/* direction helpers                                                   */
/* ------------------------------------------------------------------ */
/* Direction with polar angle (cos t, sin t) and azimuth (cos p, sin p)
 * about the axis d. */
static void rotate_dir(double d[3], double ct, double st, double cp, double sp)
{
    double u = d[0], v = d[1], w = d[2];
    double s2 = 1.0 - w * w;
    double nu, nv, nw;
    if (s2 < 1e-10) {
        nu = st * cp; nv = st * sp; nw = (w >= 0.0 ? ct : -ct);
    } else {
        double s = sqrt(s2);
        nu = u * ct + st * (u * w * cp - v * sp) / s;
        nv = v * ct + st * (v * w * cp + u * sp) / s;
        nw = w * ct - st * cp * s;
    }
    double n = sqrt(nu * nu + nv * nv + nw * nw);
    d[0] = nu / n; d[1] = nv / n; d[2] = nw / n;
}

/* Vector given in the frame whose third axis is d (same basis as rotate_dir). */
static void frame_to_lab(const double d[3], const double a[3], double out[3])
{
    double u = d[0], v = d[1], w = d[2];
    double s2 = 1.0 - w * w;
    double e1[3], e2[3];
    if (s2 < 1e-10) {
        e1[0] = 1; e1[1] = 0; e1[2] = 0; e2[0] = 0; e2[1] = 1; e2[2] = 0;
        double o0 = a[0], o1 = a[1], o2 = (w >= 0.0 ? a[2] : -a[2]);
        out[0] = o0; out[1] = o1; out[2] = o2;
        return;
    }
    double s = sqrt(s2);
    e1[0] = u * w / s; e1[1] = v * w / s; e1[2] = -s;
    e2[0] = -v / s; e2[1] = u / s; e2[2] = 0.0;
    for (int i = 0; i < 3; ++i) out[i] = a[0] * e1[i] + a[1] * e2[i] + a[2] * d[i];
    double n = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    for (int i = 0; i < 3; ++i) out[i] /= n;
}

static double mom(double T, double m) { return sqrt(T * T + 2.0 * T * m); }

/* ------------------------------------------------------------------ */
/* nuclear elastic scattering (Sec. II.A.5, Eq. 3)                     */
/* ------------------------------------------------------------------ */
/* Samples one elastic collision of a proton of kinetic energy E on (Z, A).
 * u[0]: Ranft component, u[1]: momentum transfer (or cos theta* for A = 1),
 * u[2]: azimuth.  Outputs the scattered proton's kinetic energy and lab
 * polar cosine, the recoil's kinetic energy and lab polar cosine (azimuth of
 * the recoil is the proton's + pi). */
void or_elastic_kinematics(int Z, int A, double E, const double u[3],
                           double* T1, double* cos1, double* T2, double* cos2, double* cos_cm)
{
    double M = or_nuclear_mass(Z, A);
    double m = M_PROTON;
    double plab = mom(E, m), Elab = E + m;
    double s = m * m + M * M + 2.0 * M * Elab;
    double rs = sqrt(s);
    double pcm = plab * M / rs;
    double ct;
    if (A == 1) {
        ct = 2.0 * u[1] - 1.0;
    } else {
        double a1, b1, a2, b2;
        double Ad = (double)A;
        if (A <= 62) { a1 = pow(Ad, 1.63); b1 = 14.5 * pow(Ad, 0.66); a2 = 1.4 * pow(Ad, 0.33); b2 = 10.0; }
        else { a1 = pow(Ad, 1.33); b1 = 60.0 * pow(Ad, 0.33); a2 = 0.4 * pow(Ad, 0.4); b2 = 10.0; }
        double p = pcm * 1e-3; /* GeV/c */
        double tmax = 4.0 * p * p;
        double w1 = a1 * (1.0 - exp(-b1 * tmax)) / b1;
        double w2 = a2 * (1.0 - exp(-b2 * tmax)) / b2;
        double b = (u[0] * (w1 + w2) < w1) ? b1 : b2;
        double t = -log(1.0 - u[1] * (1.0 - exp(-b * tmax))) / b; /* |t| */
        ct = 1.0 - t / (2.0 * p * p);
        if (ct < -1.0) ct = -1.0;
        if (ct > 1.0) ct = 1.0;
    }
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double beta = plab / (Elab + M), gam = (Elab + M) / rs;
    double e1 = sqrt(pcm * pcm + m * m), e2 = sqrt(pcm * pcm + M * M);
    double p1z = gam * (pcm * ct + beta * e1), p1t = pcm * st;
    double E1 = gam * (e1 + beta * pcm * ct);
    double p2z = gam * (-pcm * ct + beta * e2), p2t = pcm * st;
    double t1 = E1 - m;
    if (t1 > E) t1 = E;
    if (t1 < 0.0) t1 = 0.0;
    *T1 = t1;
    *T2 = E - t1;
    *cos1 = p1z / sqrt(p1z * p1z + p1t * p1t);
    double n2 = sqrt(p2z * p2z + p2t * p2t);
    *cos2 = n2 > 0.0 ? p2z / n2 : 1.0;
    if (cos_cm) *cos_cm = ct;
    (void)u[2];
}

/* ------------------------------------------------------------------ */
/* intranuclear cascade + evaporation (Sec. II.A.4)                    */
/* ------------------------------------------------------------------ */
#define INC_SHELLS 15
#define INC_MAX_PARTICLES 32
#define INC_MAX_RETRIES 1000
#define INC_MAX_CROSSINGS 1000
#define EVAP_MAX_STEPS 64
#define OR_MAX_PRODUCTS 160

typedef struct {
    int Z, A;
    double Rws, aws, Rout;
    double r[INC_SHELLS + 1];
    double rho_q[2][INC_SHELLS];   /* [0] neutrons, [1] protons, fm^-3 */
    double pF[2][INC_SHELLS], TF[2][INC_SHELLS], V[2][INC_SHELLS];
    double S[2];                   /* separation energies (n, p) */
} or_nucleus;

void or_nucleus_build(int Z, int A, or_nucleus* nu)
{
    memset(nu, 0, sizeof(*nu));
    nu->Z = Z; nu->A = A;
    double a13 = cbrt((double)A);
    nu->Rws = 1.16 * a13 * (1.0 - 1.16 / (a13 * a13));
    nu->aws = 0.55;
    nu->Rout = nu->Rws + nu->aws * log(99.0);
    double f[INC_SHELLS], vol[INC_SHELLS], sum = 0.0;
    for (int i = 0; i <= INC_SHELLS; ++i) nu->r[i] = nu->Rout * i / INC_SHELLS;
    for (int i = 0; i < INC_SHELLS; ++i) {
        double mid = 0.5 * (nu->r[i] + nu->r[i + 1]);
        f[i] = 1.0 / (1.0 + exp((mid - nu->Rws) / nu->aws));
        vol[i] = 4.0 / 3.0 * PI * (pow(nu->r[i + 1], 3) - pow(nu->r[i], 3));
        sum += f[i] * vol[i];
    }
    nu->S[0] = or_nuclear_mass(Z, A - 1) + M_NEUTRON - or_nuclear_mass(Z, A);
    nu->S[1] = or_nuclear_mass(Z - 1, A - 1) + M_PROTON - or_nuclear_mass(Z, A);
    for (int i = 0; i < INC_SHELLS; ++i) {
        double rho = f[i] * A / sum;
        for (int q = 0; q < 2; ++q) {
            double frac = (q == 1) ? (double)Z / A : (double)(A - Z) / A;
            double m = (q == 1) ? M_PROTON : M_NEUTRON;
            nu->rho_q[q][i] = rho * frac;
            nu->pF[q][i] = HBARC * cbrt(3.0 * PI * PI * nu->rho_q[q][i]);
            nu->TF[q][i] = sqrt(nu->pF[q][i] * nu->pF[q][i] + m * m) - m;
            nu->V[q][i] = nu->TF[q][i] + nu->S[q];
        }
    }
}

typedef struct { int species; double T; double dir[3]; } or_product; /* species: 0 n,1 p,2 d,3 t,4 He3,5 alpha */
typedef struct {
    int n; or_product p[OR_MAX_PRODUCTS];
    int Zres, Ares; double Tres, Ex_left, binding;
    int retries, transparent, collisions, overflow;
    double min_pauli_margin;   /* min over accepted collisions of (T - T_F), both products */
    double Ex_inc;             /* excitation after the cascade */
} or_event;

typedef struct { int q; double r[3], d[3], T; int shell; int done; int refl; } inc_particle;

static const int EJ_Z[6] = {0, 1, 1, 1, 2, 2};
static const int EJ_A[6] = {1, 1, 2, 3, 3, 4};
static const double EJ_G[6] = {2, 2, 3, 2, 2, 1};

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Distance along d from r to the sphere of radius R, outward root. */
static double dist_out(const double r[3], const double d[3], double R)
{
    double b = dot3(r, d), c = dot3(r, r) - R * R;
    double disc = b * b - c;
    if (disc < 0.0) disc = 0.0;
    double s = -b + sqrt(disc);
    return s > 0.0 ? s : 0.0;
}
/* Distance to the inner sphere if it is hit in front, else -1. */
static double dist_in(const double r[3], const double d[3], double R)
{
    double b = dot3(r, d);
    if (b >= 0.0) return -1.0;
    double c = dot3(r, r) - R * R;
    double disc = b * b - c;
    if (disc <= 0.0) return -1.0;
    double s = -b - sqrt(disc);
    return s > 0.0 ? s : 0.0;
}

static void iso_dir(or_stream* st, double d[3])
{
    double c = 2.0 * next_u(st) - 1.0, ph = TWO_PI * next_u(st);
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    d[0] = s * cos(ph); d[1] = s * sin(ph); d[2] = c;
}

/* Refraction or reflection of particle at a spherical boundary.  nhat is the
 * unit normal pointing into the region being entered; Vb < 0 means outside.
 * Returns 1 if it crossed. */
static int cross_boundary(inc_particle* P, const double nhat[3], double Va, double Vb, double m)
{
    double Tb = P->T - Va + Vb;
    double dn = dot3(P->d, nhat);
    if (Tb > 0.0) {
        double pa = mom(P->T, m), pb = mom(Tb, m);
        double pt2 = pa * pa * (1.0 - dn * dn);
        double pn2 = pb * pb - pt2;
        if (pn2 > 0.0) {
            double pn = sqrt(pn2), nd[3];
            for (int i = 0; i < 3; ++i) nd[i] = (pa * (P->d[i] - dn * nhat[i]) + pn * nhat[i]) / pb;
            double nn = sqrt(dot3(nd, nd));
            for (int i = 0; i < 3; ++i) P->d[i] = nd[i] / nn;
            P->T = Tb;
            return 1;
        }
    }
    for (int i = 0; i < 3; ++i) P->d[i] -= 2.0 * dn * nhat[i];
    double nn = sqrt(dot3(P->d, P->d));
    for (int i = 0; i < 3; ++i) P->d[i] /= nn;
    return 0;
}

/* Elastic NN collision, isotropic in the pair's CM frame, relativistic. */
static void nn_collide(const double p1[3], double E1, double m1, const double p2[3], double E2, double m2,
                       const double nstar[3], double p1o[3], double* T1o, double p2o[3], double* T2o)
{
    double P[3] = {p1[0] + p2[0], p1[1] + p2[1], p1[2] + p2[2]};
    double Et = E1 + E2;
    double s = Et * Et - dot3(P, P);
    double rs = sqrt(s);
    double k = sqrt(fmax(0.0, (s - (m1 + m2) * (m1 + m2)) * (s - (m1 - m2) * (m1 - m2)))) / (2.0 * rs);
    double beta[3] = {P[0] / Et, P[1] / Et, P[2] / Et};
    double b2 = dot3(beta, beta), gam = Et / rs;
    double ps[3] = {k * nstar[0], k * nstar[1], k * nstar[2]};
    double es = sqrt(k * k + m1 * m1);
    double bp = dot3(beta, ps);
    double coef = (b2 > 0.0) ? ((gam - 1.0) * bp / b2 + gam * es) : 0.0;
    for (int i = 0; i < 3; ++i) { p1o[i] = ps[i] + coef * beta[i]; p2o[i] = P[i] - p1o[i]; }
    double e1o = gam * (es + bp);
    *T1o = e1o - m1;
    *T2o = (Et - e1o) - m2;
}

/* Weisskopf-Ewing width integral I(X, a) = int_0^X (X - x) exp(2 sqrt(a x)) dx,
 * by composite Simpson quadrature in y = sqrt(x) (smooth integrand). */
double or_evap_integral(double X, double a)
{
    if (X <= 0.0) return 0.0;
    int n = 2000;
    double Y = sqrt(X), h = Y / n, s = 0.0;
    for (int i = 0; i <= n; ++i) {
        double y = i * h;
        double f = (X - y * y) * exp(2.0 * sqrt(a) * y) * 2.0 * y;
        s += f * ((i == 0 || i == n) ? 1.0 : (i % 2 ? 4.0 : 2.0));
    }
    return s * h / 3.0;
}

/* Samples z in [0, X] with density proportional to z exp(2 sqrt(a (X - z)))
 * by rejection (exact). */
static double evap_sample(or_stream* st, double X, double a, int* fallback)
{
    double sq = sqrt(a * X);
    for (int it = 0; it < 1000; ++it) {
        if (sq >= 1.0) {
            double T = sqrt(X / a);
            double u1 = next_u(st), u2 = next_u(st), u3 = next_u(st);
            double z = -T * log(u1 * u2);
            if (z > X) continue;
            if (u3 <= exp(2.0 * sqrt(a * (X - z)) - 2.0 * sq + z / T)) return z;
        } else {
            double u1 = next_u(st), u2 = next_u(st);
            double z = X * u1;
            if (u2 * X * exp(2.0 * sq) <= z * exp(2.0 * sqrt(a * (X - z)))) return z;
        }
    }
    *fallback = 1;
    return 0.5 * X;
}

/* Evaporation chain (Weisskopf-Ewing over n, p, d, t, He3, alpha) of a nucleus
 * (Z, A) with excitation Ex and momentum pc (MeV/c, Galilean with masses A u).
 * Appends products to ev and sets the final residual. */
static void evaporate(or_stream* st_, int Zc, int Ac, double Ex, double pc[3], or_event* ev)
{
    or_stream* stp = st_;
    for (int step = 0; step < EVAP_MAX_STEPS; ++step) {
        double G[6], Gs = 0.0, Sj[6], Vj[6], Xj[6];
        for (int j = 0; j < 6; ++j) {
            G[j] = 0.0;
            int Zd = Zc - EJ_Z[j], Ad = Ac - EJ_A[j];
            if (Ad < 1 || Zd < 0 || Zd > Ad) continue;
            Sj[j] = or_nuclear_mass(Zd, Ad) + or_nuclear_mass(EJ_Z[j], EJ_A[j]) - or_nuclear_mass(Zc, Ac);
            double rsum = cbrt((double)Ad) + cbrt((double)EJ_A[j]);
            Vj[j] = (EJ_Z[j] > 0 && Zd > 0) ? COULOMB_E2 * EJ_Z[j] * Zd / (1.5 * rsum) : 0.0;
            Xj[j] = Ex - Sj[j] - Vj[j];
            if (Xj[j] <= 0.0) continue;
            double mu = (double)EJ_A[j] * Ad / (EJ_A[j] + Ad);
            G[j] = EJ_G[j] * mu * (1.5 * rsum) * (1.5 * rsum) * or_evap_integral(Xj[j], Ad / 8.0);
            Gs += G[j];
        }
        if (Gs <= 0.0) break;
        double uch = next_u(stp) * Gs, acc = 0.0;
        int j = 5;
        for (int c = 0; c < 6; ++c) { acc += G[c]; if (uch < acc) { j = c; break; } }
        while (G[j] <= 0.0) --j;
        int Zd = Zc - EJ_Z[j], Ad = Ac - EJ_A[j];
        int fb = 0;
        double z = evap_sample(stp, Xj[j], Ad / 8.0, &fb);
        double eps = Vj[j] + z;                 /* kinetic energy released in the rest frame */
        double Exd = Xj[j] - z;
        double aj = EJ_A[j];
        double mu = aj * Ad / (aj + Ad) * AMU;
        double ps = sqrt(2.0 * mu * eps);
        double nd[3];
        iso_dir(stp, nd);
        double vpar[3], pej[3], pd[3];
        for (int k = 0; k < 3; ++k) {
            vpar[k] = pc[k] / (Ac * AMU);
            pej[k] = aj * AMU * vpar[k] + ps * nd[k];
            pd[k] = Ad * AMU * vpar[k] - ps * nd[k];
        }
        double pm = sqrt(dot3(pej, pej));
        or_product* o = &ev->p[ev->n++];
        o->species = j;
        o->T = dot3(pej, pej) / (2.0 * aj * AMU);
        for (int k = 0; k < 3; ++k) o->dir[k] = pej[k] / pm;
        ev->binding += Sj[j];
        Zc = Zd; Ac = Ad; Ex = Exd;
        for (int k = 0; k < 3; ++k) pc[k] = pd[k];
        if (ev->n >= OR_MAX_PRODUCTS - 1) break;
    }
    ev->Zres = Zc; ev->Ares = Ac;
    ev->Tres = dot3(pc, pc) / (2.0 * Ac * AMU);
    ev->Ex_left = Ex;
}

/* The trapped-nucleon rule of the cascade (on by default).  Off, a nucleon turned back at
 * a shell boundary keeps flying until it collides or reaches the crossing cap: the
 * untruncated reading the rule is compared with. */
static int g_trap_rule = 1;
void or_set_trap_rule(int on) { g_trap_rule = on ? 1 : 0; }

/* One non-elastic event in the frame where the incident proton moves along
 * +z.  Fills ev (products' directions in that frame). */
void or_inc_event(const or_nucleus* nu, double E, uint64_t seed, uint64_t pid, or_event* ev)
{
    or_stream st = {seed, pid, 0u, 4, {0, 0, 0, 0}};
    const double mq[2] = {M_NEUTRON, M_PROTON};
    memset(ev, 0, sizeof(*ev));
    ev->min_pauli_margin = 1e300;
    int Z = nu->Z, A = nu->A;
    double pin = mom(E, M_PROTON);
    double M_target = or_nuclear_mass(Z, A);

    inc_particle P[INC_MAX_PARTICLES];
    for (int attempt = 0; attempt < INC_MAX_RETRIES; ++attempt) {
        int n = 1, sea[2] = {A - Z, Z}, any = 0, overflow = 0, ncoll = 0;
        double margin = 1e300;
        /* entry point on the outer sphere, uniform over the projected disc */
        double b = nu->Rout * sqrt(next_u(&st)), ph = TWO_PI * next_u(&st);
        P[0].q = 1; P[0].T = E; P[0].done = 0; P[0].refl = 0;
        P[0].r[0] = b * cos(ph); P[0].r[1] = b * sin(ph);
        P[0].r[2] = -sqrt(fmax(0.0, nu->Rout * nu->Rout - b * b));
        P[0].d[0] = 0; P[0].d[1] = 0; P[0].d[2] = 1;
        {
            double rr = sqrt(dot3(P[0].r, P[0].r));
            double nh[3] = {-P[0].r[0] / rr, -P[0].r[1] / rr, -P[0].r[2] / rr};
            cross_boundary(&P[0], nh, 0.0, nu->V[1][INC_SHELLS - 1], M_PROTON);
            P[0].shell = INC_SHELLS - 1;
        }
        int esc_idx[INC_MAX_PARTICLES], n_esc = 0;
        for (int ip = 0; ip < n; ++ip) {
            inc_particle* p = &P[ip];
            int q = p->q, crossings = 0, iters = 0;
            double m = mq[q];
            for (;;) {
                int i = p->shell;
                if (p->T - nu->V[q][i] <= 0.0) { p->done = 2; break; }   /* bound: captured */
                if (++iters > 100000) { p->done = 2; break; }             /* flight cap: captured */
                double s_out = dist_out(p->r, p->d, nu->r[i + 1]);
                double s_in = (i > 0) ? dist_in(p->r, p->d, nu->r[i]) : -1.0;
                int inner = (s_in >= 0.0 && s_in < s_out);
                double s_b = inner ? s_in : s_out;
                double sig_like = or_sigma_nn(p->T, 1) * FM2_PER_MB;
                double sig_unlike = or_sigma_nn(p->T, 0) * FM2_PER_MB;
                double sig_p = (q == 1) ? sig_like : sig_unlike;
                double sig_n = (q == 0) ? sig_like : sig_unlike;
                double rate_p = sea[1] > 0 ? nu->rho_q[1][i] * sig_p : 0.0;
                double rate_n = sea[0] > 0 ? nu->rho_q[0][i] * sig_n : 0.0;
                double rate = rate_p + rate_n;
                double uc = next_u(&st);
                double s_c = rate > 0.0 ? -log(uc) / rate : 1e300;
                if (s_c < s_b) {
                    for (int k = 0; k < 3; ++k) p->r[k] += s_c * p->d[k];
                    int q2 = (next_u(&st) * rate < rate_p) ? 1 : 0;
                    double m2 = mq[q2];
                    double p2m = nu->pF[q2][i] * cbrt(next_u(&st));
                    double d2[3];
                    iso_dir(&st, d2);
                    double ns[3];
                    iso_dir(&st, ns);
                    double p1v[3], p2v[3], p1o[3], p2o[3], T1o, T2o;
                    double p1m = mom(p->T, m);
                    for (int k = 0; k < 3; ++k) { p1v[k] = p1m * p->d[k]; p2v[k] = p2m * d2[k]; }
                    nn_collide(p1v, p->T + m, m, p2v, sqrt(p2m * p2m + m2 * m2), m2, ns, p1o, &T1o, p2o, &T2o);
                    if (T1o < nu->TF[q][i] || T2o < nu->TF[q2][i]) continue;        /* Pauli blocked */
                    if (n >= INC_MAX_PARTICLES) { overflow++; continue; }            /* stack full: blocked */
                    double mg = fmin(T1o - nu->TF[q][i], T2o - nu->TF[q2][i]);
                    if (mg < margin) margin = mg;
                    double n1 = sqrt(dot3(p1o, p1o)), n2 = sqrt(dot3(p2o, p2o));
                    for (int k = 0; k < 3; ++k) { p->d[k] = p1o[k] / n1; }
                    p->T = T1o;
                    p->refl = 0;
                    inc_particle* c = &P[n++];
                    c->q = q2; c->T = T2o; c->shell = i; c->done = 0; c->refl = 0;
                    for (int k = 0; k < 3; ++k) { c->r[k] = p->r[k]; c->d[k] = p2o[k] / n2; }
                    sea[q2]--;
                    any = 1; ncoll++;
                    p = &P[ip];
                } else {
                    for (int k = 0; k < 3; ++k) p->r[k] += s_b * p->d[k];
                    if (++crossings > INC_MAX_CROSSINGS) { p->done = 2; break; }
                    double rr = sqrt(dot3(p->r, p->r));
                    double nh[3];
                    if (inner) {
                        for (int k = 0; k < 3; ++k) nh[k] = -p->r[k] / rr;
                        if (cross_boundary(p, nh, nu->V[q][i], nu->V[q][i - 1], m)) p->shell = i - 1;
                        else if (++p->refl >= 2 && g_trap_rule) { p->done = 2; break; }
                    } else {
                        for (int k = 0; k < 3; ++k) nh[k] = p->r[k] / rr;
                        double Vb = (i + 1 < INC_SHELLS) ? nu->V[q][i + 1] : 0.0;
                        if (cross_boundary(p, nh, nu->V[q][i], Vb, m)) {
                            if (i + 1 == INC_SHELLS) { p->done = 1; break; }   /* escaped */
                            p->shell = i + 1;
                        } else if (++p->refl >= 2 && g_trap_rule) {
                            /* between collisions energy and angular momentum are conserved, so
                             * a nucleon turned back once can never reach the surface; on its
                             * second turn without an allowed collision it is trapped */
                            p->done = 2;
                            break;
                        }
                    }
                }
            }
            if (p->done == 1) esc_idx[n_esc++] = ip;
        }
        if (!any) { ev->retries++; continue; }
        /* residual nucleus and excitation from energy and momentum conservation */
        int zesc = 0;
        double sumT = 0.0, prec[3] = {0.0, 0.0, pin};
        for (int k = 0; k < n_esc; ++k) {
            inc_particle* p = &P[esc_idx[k]];
            zesc += p->q;
            sumT += p->T;
            double pm = mom(p->T, mq[p->q]);
            for (int j = 0; j < 3; ++j) prec[j] -= pm * p->d[j];
        }
        int Zr = Z + 1 - zesc, Ar = A + 1 - n_esc;
        if (Ar < 1 || Zr < 0 || Zr > Ar) { ev->retries++; continue; }
        double dM = or_nuclear_mass(Zr, Ar) - M_target - M_PROTON;
        for (int k = 0; k < n_esc; ++k) dM += mq[P[esc_idx[k]].q];
        double Trec = dot3(prec, prec) / (2.0 * Ar * AMU);
        double Ex = E - sumT - Trec - dM;
        if (Ex < 0.0) { ev->retries++; continue; }
        /* accepted */
        ev->collisions = ncoll; ev->overflow = overflow; ev->min_pauli_margin = margin;
        ev->binding = dM; ev->Ex_inc = Ex;
        for (int k = 0; k < n_esc; ++k) {
            inc_particle* p = &P[esc_idx[k]];
            or_product* o = &ev->p[ev->n++];
            o->species = p->q; o->T = p->T;
            for (int j = 0; j < 3; ++j) o->dir[j] = p->d[j];
        }
        {
            double pc[3] = {prec[0], prec[1], prec[2]};
            evaporate(&st, Zr, Ar, Ex, pc, ev);
        }
        return;
    }
    ev->transparent = 1;
}

/* ------------------------------------------------------------------ */
/* the transporter                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
    double ZA, I_eV, f, X0mass;
    int cls;                         /* range table used */
    double n_per_g[OR_MAX_NUC_PER_MAT];
} or_matinfo;

typedef struct {
    const or_problem* P;
    uint64_t seed;
    or_matinfo* mi;
    or_range_table* tables;          /* [0] water reference, then one per own-table material */
    or_nucleus* nuclei;              /* per nuclide */
    double* tally;                   /* [V][B] */
    double* hl;                      /* per-history ledger [h][4] or NULL */
    or_totals* tot;
    double* esc;                     /* escaping protons [cap][8]: E, x, y, z, u, v, w, root */
    long esc_cap, esc_n;
    double* let_num;                 /* [V][B] sum of e * L (MeV keV/um) over proton energy losses, or NULL */
    double* let_den;                 /* [V][B] sum of e (MeV) over the same deposits */
} or_ctx;

typedef struct { double x[3], d[3], E, nmfp; int iv[3]; uint64_t pid; uint64_t root; } or_particle;

typedef struct { or_particle* a; int n, cap; } or_pstack;
static void push(or_pstack* s, const or_particle* p)
{
    if (s->n == s->cap) { s->cap = s->cap ? 2 * s->cap : 64; s->a = (or_particle*)realloc(s->a, sizeof(or_particle) * s->cap); }
    s->a[s->n++] = *p;
}

static void voxel_props(const or_ctx* c, const int iv[3], int* m, double* rho)
{
    const or_problem* P = c->P;
    long v = ((long)iv[2] * P->ny + iv[1]) * P->nx + iv[0];
    if (P->hu_vol) {
        int hu = P->hu_vol[v];
        int b = P->n_hu - 1;
        for (int k = 0; k < P->n_hu; ++k) if (hu >= P->hu[k].lo && hu < P->hu[k].hi) { b = k; break; }
        if (hu < P->hu[0].lo) b = 0;
        *m = P->hu[b].material;
        *rho = P->hu[b].rho_a + P->hu[b].rho_b * hu;
    } else {
        *m = P->mat_vol[v];
        *rho = (double)P->rho_vol[v];
    }
}

static void deposit(or_ctx* c, const int iv[3], uint64_t root, double e)
{
    const or_problem* P = c->P;
    long v = ((long)iv[2] * P->ny + iv[1]) * P->nx + iv[0];
    c->tally[v * P->n_batches + (long)(root % (uint64_t)P->n_batches)] += e;
    c->tot->deposited += e;
    if (c->hl) c->hl[root * 4 + 1] += e;
}
/* Dose-averaged LET (Sec. IV): each energy loss e of a transported proton, with the
 * mean CSDA stopping power L of the local medium over the path that lost it (MeV/cm,
 * scored in keV/um = 0.1 MeV/cm).  Recoil nuclei and fragments do not score. */
static void score_let(or_ctx* c, const int iv[3], uint64_t root, double e, double L_mev_cm)
{
    if (!c->let_num) return;
    const or_problem* P = c->P;
    long v = ((long)iv[2] * P->ny + iv[1]) * P->nx + iv[0];
    long i = v * P->n_batches + (long)(root % (uint64_t)P->n_batches);
    c->let_num[i] += e * (0.1 * L_mev_cm);
    c->let_den[i] += e;
}
static void escape(or_ctx* c, uint64_t root, double e)
{
    c->tot->escaped += e;
    if (c->hl) c->hl[root * 4 + 2] += e;
}
static void bind_energy(or_ctx* c, uint64_t root, double e)
{
    c->tot->binding += e;
    if (c->hl) c->hl[root * 4 + 3] += e;
}

static double sigma_per_gram(const or_ctx* c, int m, double E, int channel /* 0 inel, 1 el, 2 both */)
{
    const or_material* M = &c->P->mat[m];
    double s = 0.0;
    for (int k = 0; k < M->n; ++k) {
        const or_nuclide* nu = &c->P->nuc[M->nuc[k]];
        double sg = 0.0;
        if (channel != 1 && !(c->P->flags & OR_NO_INELASTIC)) sg += or_sigma_inelastic(nu->Z, nu->A, E);
        if (channel != 0 && !(c->P->flags & OR_NO_ELASTIC)) sg += or_sigma_elastic(nu->Z, nu->A, E);
        s += c->mi[m].n_per_g[k] * sg * MB_TO_CM2;
    }
    return s;
}

/* Distance to the faces of voxel iv along d; axis and direction of exit. */
static double voxel_exit(const or_problem* P, const double x[3], const double d[3], const int iv[3], int* axis)
{
    const double lo[3] = {P->x0, P->y0, P->z0}, w[3] = {P->dx, P->dy, P->dz};
    double best = 1e300;
    *axis = 0;
    for (int a = 0; a < 3; ++a) {
        double s;
        if (d[a] > 0.0) s = (lo[a] + (iv[a] + 1) * w[a] - x[a]) / d[a];
        else if (d[a] < 0.0) s = (lo[a] + iv[a] * w[a] - x[a]) / d[a];
        else continue;
        if (s < 0.0) s = 0.0;
        if (s < best) { best = s; *axis = a; }
    }
    return best;
}

static void new_particle(or_pstack* st, uint64_t seed, uint64_t parent, uint32_t idx, uint64_t root,
                         const double x[3], const double d[3], double T, const int iv[3], or_totals* tot)
{
    or_particle q;
    q.pid = child_pid(seed, parent, idx);
    q.root = root;
    for (int k = 0; k < 3; ++k) { q.x[k] = x[k]; q.d[k] = d[k]; q.iv[k] = iv[k]; }
    q.E = T;
    double u[4];
    draw4(seed, q.pid, 1u, 4u, u);
    q.nmfp = -log(u[0]);
    push(st, &q);
    tot->secondaries += 1.0;
}

static void nonelastic(or_ctx* c, or_particle* p, int nuc, or_pstack* st)
{
    const or_problem* P = c->P;
    or_event ev;
    or_inc_event(&c->nuclei[nuc], p->E, c->seed, p->pid, &ev);
    c->tot->inc_retries += ev.retries;
    if (ev.transparent) {
        c->tot->transparent += 1.0;
        new_particle(st, c->seed, p->pid, 0x20000u, p->root, p->x, p->d, p->E, p->iv, c->tot);
        return;
    }
    for (int k = 0; k < ev.n; ++k) {
        const or_product* o = &ev.p[k];
        if (o->species == 1) {
            if (o->T > E_CUT) {
                double dl[3];
                frame_to_lab(p->d, o->dir, dl);
                new_particle(st, c->seed, p->pid, (uint32_t)k, p->root, p->x, dl, o->T, p->iv, c->tot);
            } else deposit(c, p->iv, p->root, o->T);
        } else if (o->species == 0) escape(c, p->root, o->T);
        else deposit(c, p->iv, p->root, o->T);
    }
    deposit(c, p->iv, p->root, ev.Tres);
    escape(c, p->root, ev.Ex_left);
    bind_energy(c, p->root, ev.binding);
    (void)P;
}

/* Transport of one proton until it stops, leaves the grid or is absorbed in a
 * non-elastic event (Sec. II.A.3). */
static void transport_one(or_ctx* c, or_particle* p, or_pstack* st)
{
    const or_problem* P = c->P;
    const int dims[3] = {P->nx, P->ny, P->nz};
    uint32_t k = 0;
    for (;;) {
        if (p->E <= E_CUT) {
            deposit(c, p->iv, p->root, p->E);
            if (c->let_num && p->E > 0.0) {   /* absorbed over its residual range */
                int m0; double rho0;
                voxel_props(c, p->iv, &m0, &rho0);
                const or_matinfo* m0i = &c->mi[m0];
                double R0 = range_of_energy(&c->tables[m0i->cls], p->E) / (rho0 * m0i->f);
                if (R0 > 0.0) score_let(c, p->iv, p->root, p->E, p->E / R0);
            }
            return;
        }
        if (k >= 100000u) { deposit(c, p->iv, p->root, p->E); c->tot->errors += 1.0; return; }
        int m; double rho;
        voxel_props(c, p->iv, &m, &rho);
        const or_matinfo* mi = &c->mi[m];
        const or_range_table* rt = &c->tables[mi->cls];
        double E0 = p->E;
        double Rm = range_of_energy(rt, E0);
        double rf = rho * mi->f;
        double Rcm = Rm / rf;
        double sig_in = sigma_per_gram(c, m, E0, 0) * rho;
        double sig_el = sigma_per_gram(c, m, E0, 1) * rho;
        double sig = sig_in + sig_el;
        double lam = sig > 0.0 ? p->nmfp / sig : 1e300;
        int axis;
        double d = voxel_exit(P, p->x, p->d, p->iv, &axis);
        c->tot->steps += 1.0;
        if (Rcm <= lam && Rcm <= d) {
            deposit(c, p->iv, p->root, E0);
            if (Rcm > 0.0) score_let(c, p->iv, p->root, E0, E0 / Rcm);
            return;
        }
        int nuclear = (lam <= d);
        double dx = nuclear ? lam : d;
        double ua[5];
        step_uniforms(c->seed, p->pid, k, ua);
        double tau = ua[4];
        double x1[3];
        for (int a = 0; a < 3; ++a) x1[a] = p->x[a] + tau * dx * p->d[a];
        if (!(P->flags & OR_NO_MCS) && (P->flags & OR_MOLIERE)) {
            double chic2, B;
            or_moliere_params(P, m, E0, dx * rho, &chic2, &B);
            double th = or_moliere_theta(ua[0], chic2, B);
            if (th > 0.0) rotate_dir(p->d, cos(th), sin(th), cos(TWO_PI * ua[1]), sin(TWO_PI * ua[1]));
        } else if (!(P->flags & OR_NO_MCS)) {
            double th0 = or_highland_theta0(E0, dx, mi->X0mass / rho);
            double r = sqrt(-2.0 * log(ua[0]));
            double tx = th0 * r * cos(TWO_PI * ua[1]), ty = th0 * r * sin(TWO_PI * ua[1]);
            double th = sqrt(tx * tx + ty * ty);
            if (th > 0.0) rotate_dir(p->d, cos(th), sin(th), tx / th, ty / th);
        }
        double L2 = (1.0 - tau) * dx;
        int axis2;
        double d2 = voxel_exit(P, x1, p->d, p->iv, &axis2);
        int crossing = 0;
        if (d2 <= L2) { L2 = d2; crossing = 1; nuclear = 0; }
        double s = tau * dx + L2;
        for (int a = 0; a < 3; ++a) p->x[a] = x1[a] + L2 * p->d[a];
        double Rleft = Rm - s * rf;
        double dE = (Rleft > 0.0) ? E0 - energy_of_range(rt, Rleft) : E0;
        const double L_step = s > 0.0 ? dE / s : 0.0;     /* mean CSDA stopping power over the path */
        if (!(P->flags & OR_NO_STRAGGLING)) {
            double xi = 0.0, kap = 1e300;
            if ((P->flags & OR_VAVILOV) && or_vav_ready) or_vavilov_params(E0, rho, mi->ZA, s, &xi, &kap);
            if (kap <= 10.0) {
                double g = 1.0 + E0 / M_PROTON;
                dE += xi * or_vavilov_z(kap, 1.0 - 1.0 / (g * g), ua[2]);
            } else {
                double var = or_bohr_variance(E0, rho, mi->ZA, s);
                dE += sqrt(var) * sqrt(-2.0 * log(ua[2])) * cos(TWO_PI * ua[3]);
            }
        }
        if (dE < 0.0) dE = 0.0;
        if (dE > E0) dE = E0;
        deposit(c, p->iv, p->root, dE);
        score_let(c, p->iv, p->root, dE, L_step);
        p->E = E0 - dE;
        p->nmfp -= sig * s;
        ++k;
        if (crossing) {
            int a = axis2;
            p->iv[a] += (p->d[a] > 0.0) ? 1 : -1;
            if (p->iv[a] < 0 || p->iv[a] >= dims[a]) {
                escape(c, p->root, p->E);
                if (c->esc && c->esc_n < c->esc_cap) {
                    double* o = c->esc + c->esc_n++ * 8;
                    o[0] = p->E; o[1] = p->x[0]; o[2] = p->x[1]; o[3] = p->x[2];
                    o[4] = p->d[0]; o[5] = p->d[1]; o[6] = p->d[2]; o[7] = (double)p->root;
                }
                return;
            }
        } else if (nuclear && p->E > E_CUT) {
            /* channel and target from the step-start cross-sections */
            const or_material* M = &P->mat[m];
            double ub[4];
            draw4(c->seed, p->pid, k - 1, 1u, ub);
            int inel = (ub[0] * sig < sig_in);
            double part[OR_MAX_NUC_PER_MAT], tot = 0.0;
            for (int j = 0; j < M->n; ++j) {
                const or_nuclide* nu = &P->nuc[M->nuc[j]];
                double sg = inel ? (P->flags & OR_NO_INELASTIC ? 0.0 : or_sigma_inelastic(nu->Z, nu->A, E0))
                                 : (P->flags & OR_NO_ELASTIC ? 0.0 : or_sigma_elastic(nu->Z, nu->A, E0));
                part[j] = mi->n_per_g[j] * sg;
                tot += part[j];
            }
            int t = M->n - 1;
            double acc = 0.0, ut = ub[1] * tot;
            for (int j = 0; j < M->n; ++j) { acc += part[j]; if (ut < acc) { t = j; break; } }
            while (t > 0 && part[t] <= 0.0) --t;
            int nuc = M->nuc[t];
            const or_nuclide* nu = &P->nuc[nuc];
            if (inel) {
                c->tot->inelastic += 1.0;
                nonelastic(c, p, nuc, st);
                return;
            }
            c->tot->elastic += 1.0;
            double ue[4];
            draw4(c->seed, p->pid, k - 1, 2u, ue);
            double T1, c1, T2, c2;
            or_elastic_kinematics(nu->Z, nu->A, p->E, ue, &T1, &c1, &T2, &c2, NULL);
            double ph = TWO_PI * ue[2];
            double cp = cos(ph), sp = sin(ph);
            double din[3] = {p->d[0], p->d[1], p->d[2]};
            rotate_dir(p->d, c1, sqrt(fmax(0.0, 1.0 - c1 * c1)), cp, sp);
            if (nu->A == 1) {
                if (T2 > E_CUT) {
                    double d2v[3] = {din[0], din[1], din[2]};
                    rotate_dir(d2v, c2, sqrt(fmax(0.0, 1.0 - c2 * c2)), -cp, -sp);
                    new_particle(st, c->seed, p->pid, 0x10000u + (k - 1), p->root, p->x, d2v, T2, p->iv, c->tot);
                } else deposit(c, p->iv, p->root, T2);
            } else deposit(c, p->iv, p->root, T2);
            p->E = T1;
            p->nmfp = -log(ub[2]);
        }
    }
}

/* Histories allocated to spots in proportion to weight, largest remainder
 * (ties to the lower index). */
static void allocate_histories(const or_problem* P, uint64_t n, uint64_t* cnt)
{
    double W = 0.0;
    for (int s = 0; s < P->n_spots; ++s) W += P->spots[s].weight;
    uint64_t used = 0;
    double* rem = (double*)malloc(sizeof(double) * (P->n_spots > 0 ? P->n_spots : 1));
    for (int s = 0; s < P->n_spots; ++s) {
        double q = (double)n * P->spots[s].weight / W;
        cnt[s] = (uint64_t)floor(q);
        rem[s] = q - floor(q);
        used += cnt[s];
    }
    while (used < n) {
        int best = 0;
        for (int s = 1; s < P->n_spots; ++s) if (rem[s] > rem[best]) best = s;
        cnt[best]++; rem[best] = -1.0; used++;
    }
    free(rem);
}

void or_allocate_histories(const or_problem* P, uint64_t n, uint64_t* cnt) { allocate_histories(P, n, cnt); }

int or_material_info(const or_problem* P, int m, double* out /* ZA, I, f, X0mass, cls */)
{
    const or_material* M = &P->mat[m];
    double ZA = 0.0, lnI = 0.0, inv = 0.0;
    for (int k = 0; k < M->n; ++k) {
        const or_nuclide* nu = &P->nuc[M->nuc[k]];
        ZA += M->w[k] * nu->Z / nu->mass_u;
        inv += M->w[k] / or_radiation_length_element(nu->Z, nu->mass_u);
    }
    for (int k = 0; k < M->n; ++k) {
        const or_nuclide* nu = &P->nuc[M->nuc[k]];
        lnI += M->w[k] * nu->Z / nu->mass_u * log(nu->I_eV);
    }
    double I = M->I_eV > 0.0 ? M->I_eV : exp(lnI / ZA);
    out[0] = ZA; out[1] = I; out[3] = 1.0 / inv;
    /* Eq. 1 scaling factor: ratio of mass stopping powers to water at 100 MeV */
    if (M->own_table || m == 0) out[2] = 1.0;
    else {
        double w[5];
        or_material_info(P, 0, w);
        out[2] = or_mass_stopping_power(100.0, ZA, I) / or_mass_stopping_power(100.0, w[0], w[1]);
    }
    return 0;
}

/* Runs histories [h_begin, h_end) of an n_hist-history simulation. */
int or_run_full(const or_problem* P, uint64_t n_hist, uint64_t h_begin, uint64_t h_end, uint64_t seed,
                double* tally, double* hist_ledger, or_totals* tot, double* esc, long esc_cap, long* esc_n,
                double* let_num, double* let_den)
{
    if (!P || P->n_mat < 1 || P->n_spots < 1 || P->n_batches < 1) return -1;
    if ((let_num == NULL) != (let_den == NULL)) return -1;
    or_ctx c;
    memset(&c, 0, sizeof(c));
    memset(tot, 0, sizeof(*tot));
    c.P = P; c.seed = seed; c.tally = tally; c.hl = hist_ledger; c.tot = tot;
    c.esc = esc; c.esc_cap = esc_cap; c.esc_n = 0;
    c.let_num = let_num; c.let_den = let_den;
    c.mi = (or_matinfo*)calloc(P->n_mat, sizeof(or_matinfo));
    c.tables = (or_range_table*)calloc(P->n_mat + 1, sizeof(or_range_table));
    int ncls = 1;
    for (int m = 0; m < P->n_mat; ++m) {
        double info[5];
        or_material_info(P, m, info);
        c.mi[m].ZA = info[0]; c.mi[m].I_eV = info[1]; c.mi[m].f = info[2]; c.mi[m].X0mass = info[3];
        for (int k = 0; k < P->mat[m].n; ++k)
            c.mi[m].n_per_g[k] = P->mat[m].w[k] * N_AVOGADRO / P->nuc[P->mat[m].nuc[k]].mass_u;
        if (m == 0) { c.mi[m].cls = 0; range_table_build(&c.tables[0], info[0], info[1]); }
        else if (P->mat[m].own_table) { c.mi[m].cls = ncls; range_table_build(&c.tables[ncls], info[0], info[1]); ncls++; }
        else c.mi[m].cls = 0;
    }
    c.nuclei = (or_nucleus*)calloc(P->n_nuc, sizeof(or_nucleus));
    for (int i = 0; i < P->n_nuc; ++i)
        if (P->nuc[i].A >= 2) or_nucleus_build(P->nuc[i].Z, P->nuc[i].A, &c.nuclei[i]);

    uint64_t* cnt = (uint64_t*)calloc(P->n_spots, sizeof(uint64_t));
    allocate_histories(P, n_hist, cnt);
    or_pstack st = {NULL, 0, 0};
    int s = 0;
    uint64_t first = 0;
    for (uint64_t h = h_begin; h < h_end && h < n_hist; ++h) {
        while (h >= first + cnt[s]) { first += cnt[s]; ++s; }
        const or_spot* sp = &P->spots[s];
        double u[4];
        draw4(seed, h, 0u, 4u, u);
        or_particle p;
        p.pid = h; p.root = h;
        double r = sqrt(-2.0 * log(u[0]));
        p.x[0] = sp->x + sp->sigma_x * r * cos(TWO_PI * u[1]);
        p.x[1] = sp->y + sp->sigma_y * r * sin(TWO_PI * u[1]);
        p.x[2] = P->z0;
        p.E = sp->E + sp->sigma_E * sqrt(-2.0 * log(u[2])) * cos(TWO_PI * u[3]);
        if (p.E < 0.0) p.E = 0.0;
        double dn = sqrt(sp->u * sp->u + sp->v * sp->v + sp->w * sp->w);
        p.d[0] = sp->u / dn; p.d[1] = sp->v / dn; p.d[2] = sp->w / dn;
        draw4(seed, h, 1u, 4u, u);
        p.nmfp = -log(u[0]);
        tot->incident += p.E;
        if (hist_ledger) hist_ledger[h * 4 + 0] += p.E;
        p.iv[0] = (int)floor((p.x[0] - P->x0) / P->dx);
        p.iv[1] = (int)floor((p.x[1] - P->y0) / P->dy);
        p.iv[2] = 0;
        if (p.iv[0] < 0 || p.iv[0] >= P->nx || p.iv[1] < 0 || p.iv[1] >= P->ny || p.d[2] <= 0.0) {
            escape(&c, h, p.E);
            continue;
        }
        st.n = 0;
        push(&st, &p);
        while (st.n > 0) {
            or_particle q = st.a[--st.n];
            transport_one(&c, &q, &st);
        }
    }
    free(st.a); free(cnt); free(c.nuclei); free(c.tables); free(c.mi);
    if (esc_n) *esc_n = c.esc_n;
    return 0;
}

int or_run_esc(const or_problem* P, uint64_t n_hist, uint64_t h_begin, uint64_t h_end, uint64_t seed,
               double* tally, double* hist_ledger, or_totals* tot, double* esc, long esc_cap, long* esc_n)
{
    return or_run_full(P, n_hist, h_begin, h_end, seed, tally, hist_ledger, tot, esc, esc_cap, esc_n, NULL, NULL);
}

int or_run(const or_problem* P, uint64_t n_hist, uint64_t h_begin, uint64_t h_end, uint64_t seed,
           double* tally, double* hist_ledger, or_totals* tot)
{
    return or_run_esc(P, n_hist, h_begin, h_end, seed, tally, hist_ledger, tot, NULL, 0, NULL);
}

/* Small helpers exposed for the pin tests. */
double or_range_csda(const or_problem* P, int m, double E)
{
    double info[5];
    or_material_info(P, m, info);
    or_range_table* t = (or_range_table*)malloc(sizeof(or_range_table));
    range_table_build(t, info[0], info[1]);
    double r = range_of_energy(t, E);
    free(t);
    return r;
}

int or_range_roundtrip(double ZA, double I_eV, int n, const double* E, double* R, double* Eback)
{
    or_range_table* t = (or_range_table*)malloc(sizeof(or_range_table));
    range_table_build(t, ZA, I_eV);
    for (int i = 0; i < n; ++i) { R[i] = range_of_energy(t, E[i]); Eback[i] = energy_of_range(t, R[i]); }
    free(t);
    return 0;
}

void or_draw4(uint64_t seed, uint64_t pid, uint32_t word2, uint32_t tag, double u[4]) { draw4(seed, pid, word2, tag, u); }
uint64_t or_child_pid(uint64_t seed, uint64_t pid, uint32_t idx) { return child_pid(seed, pid, idx); }

/* Runs n events at energy E on (Z, A) with pids pid0 + i; writes per event
 * summary rows and per product rows.  summary: [n][8] = n_products, Zres,
 * Ares, Tres, Ex_left, binding, retries, transparent.  products: [n][cap][5]
 * = species, T, dx, dy, dz (rows past n_products untouched). */
int or_inc_batch(int Z, int A, double E, uint64_t seed, uint64_t pid0, int n, int cap,
                 double* summary, double* products, double* extra /* [n][3]: collisions, min margin, Ex_inc */)
{
    or_nucleus nu;
    or_nucleus_build(Z, A, &nu);
    or_event* ev = (or_event*)malloc(sizeof(or_event));
    for (int i = 0; i < n; ++i) {
        or_inc_event(&nu, E, seed, pid0 + (uint64_t)i, ev);
        double* s = summary + (size_t)i * 8;
        s[0] = ev->n; s[1] = ev->Zres; s[2] = ev->Ares; s[3] = ev->Tres; s[4] = ev->Ex_left;
        s[5] = ev->binding; s[6] = ev->retries; s[7] = ev->transparent;
        if (extra) { extra[i * 3] = ev->collisions; extra[i * 3 + 1] = ev->min_pauli_margin; extra[i * 3 + 2] = ev->Ex_inc; }
        for (int k = 0; k < ev->n && k < cap; ++k) {
            double* o = products + ((size_t)i * cap + k) * 5;
            o[0] = ev->p[k].species; o[1] = ev->p[k].T;
            o[2] = ev->p[k].dir[0]; o[3] = ev->p[k].dir[1]; o[4] = ev->p[k].dir[2];
        }
    }
    free(ev);
    return 0;
}

int or_nucleus_info(int Z, int A, double* out /* Rout, S_n, S_p, then r[16], rho_p[15], rho_n[15], TF_p[15], TF_n[15], V_p[15], V_n[15] */)
{
    or_nucleus nu;
    or_nucleus_build(Z, A, &nu);
    out[0] = nu.Rout; out[1] = nu.S[0]; out[2] = nu.S[1];
    double* o = out + 3;
    for (int i = 0; i <= INC_SHELLS; ++i) *o++ = nu.r[i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.rho_q[1][i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.rho_q[0][i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.TF[1][i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.TF[0][i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.V[1][i];
    for (int i = 0; i < INC_SHELLS; ++i) *o++ = nu.V[0][i];
    return 0;
}

/* Evaporation sampler exposed for the distribution pin: n samples. */
int or_evap_sample_batch(double X, double a, uint64_t seed, uint64_t pid, int n, double* z)
{
    or_stream st = {seed, pid, 0u, 4, {0, 0, 0, 0}};
    for (int i = 0; i < n; ++i) { int fb = 0; z[i] = evap_sample(&st, X, a, &fb); }
    return 0;
}

/* Batch statistics of Sec. II.B.2: total and its standard error from B group tallies. */
int or_batch_stats(const double* tally, long n_vox, int B, double* total, double* sigma)
{
    for (long v = 0; v < n_vox; ++v) {
        double s = 0.0;
        for (int b = 0; b < B; ++b) s += tally[v * B + b];
        double mean = s / B, ss = 0.0;
        for (int b = 0; b < B; ++b) { double d = tally[v * B + b] - mean; ss += d * d; }
        total[v] = s;
        sigma[v] = (B > 1) ? sqrt((double)B / (B - 1) * ss) : 0.0;
    }
    return 0;
}

/* Evaporation of a nucleus at rest, for the isotropy and branching pins.
 * out: [n][4] = species of the first emission (-1 if none), its T, cos theta, n_products. */
int or_evap_batch(int Z, int A, double Ex, uint64_t seed, uint64_t pid0, int n, double* out)
{
    or_event* ev = (or_event*)malloc(sizeof(or_event));
    for (int i = 0; i < n; ++i) {
        or_stream st = {seed, pid0 + (uint64_t)i, 0u, 4, {0, 0, 0, 0}};
        memset(ev, 0, sizeof(*ev));
        double pc[3] = {0.0, 0.0, 0.0};
        evaporate(&st, Z, A, Ex, pc, ev);
        double* o = out + (size_t)i * 4;
        if (ev->n > 0) { o[0] = ev->p[0].species; o[1] = ev->p[0].T; o[2] = ev->p[0].dir[2]; }
        else { o[0] = -1; o[1] = 0; o[2] = 0; }
        o[3] = ev->n;
    }
    free(ev);
    return 0;
}
