// mra_device.cuh -- device building blocks shared by the M-RA kernels.
//
// FP64 tile arithmetic for one CTA of NT threads: covariance tiles (Sec. 2.1,
// Eq. mat15), region boxes and knots (Sec. 2.2), a register-blocked tile
// product staged through shared memory, and in-shared-memory Cholesky and
// triangular inversion.  On GB300 the FP64 pipe retires 2 DFMA per clock per
// SM, so every routine here is written to keep DFMA lanes busy with useful
// work; shared-memory bandwidth is never the limit.
#pragma once
#include <cmath>
#include <cstring>
#include <cstdint>
#include <cuda_runtime.h>

namespace mra {

constexpr int NT = 256;          // threads per CTA for every kernel
constexpr int KC = 32;           // k-chunk of the staged tile product
constexpr int MAX_R_DEV = 64;    // largest r (knots per internal region)
constexpr double SQRT3 = 1.7320508075688772935;
constexpr double PI = 3.141592653589793238463;

// ---- error status (device) ------------------------------------------------
// status[0] = first error code, status[1] = level, status[2] = region
enum : int { ST_OK = 0, ST_NOT_PD = 4, ST_LIMIT = 6, ST_ARG = 1, ST_TIMEOUT = 7 };

__device__ __forceinline__ void flag_error(int* status, int code, int level, long region) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = level;
    status[2] = (int)region;
  }
}

// ---- covariance function C0 (Sec. 2.1; Eq. mat15; nonstationary variance) --
struct Cov {
  double sigma2, kappa;
  int family;   // 0 exponential, 1 Matern-1.5, 2 Matern of smoothness nu
  int nonstat;
  double ik;    // 1 / kappa (set by make_cov)
  // family 2 (set by make_cov): nu, sqrt(2 nu), log of 2^(1-nu) / Gamma(nu) and
  // its derivative in nu, -log 2 - digamma(nu)
  double nu, snu, lcnu, dlcnu;
};

// digamma(x), x > 0, for the host: psi(x) = psi(x + k) - sum_{j<k} 1/(x + j) with
// x + k >= 8, then the asymptotic series of psi (Abramowitz & Stegun 6.3.18):
// log y - 1/(2y) - sum_{n>=1} B_2n / (2n y^2n), B_2..B_12 = 1/6, -1/30, 1/42,
// -1/30, 5/66, -691/2730 (truncation below 1e-17 at y >= 8).
inline double digamma_host(double x) {
  double acc = 0.0;
  while (x < 8.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double y2 = 1.0 / (x * x);
  const double series = y2 * (1.0 / 12 - y2 * (1.0 / 120 - y2 * (1.0 / 252 - y2 * (1.0 / 240 - y2 * (1.0 / 132 -
                                                                                                   y2 * 691.0 / 32760)))));
  return acc + std::log(x) - 0.5 / x - series;
}

inline Cov make_cov(double sigma2, double kappa, int family, int nonstat, double nu = 0.0) {
  Cov c{sigma2, kappa, family, nonstat, 1.0 / kappa, nu, 0.0, 0.0, 0.0};
  if (family == 2) {
    c.snu = std::sqrt(2.0 * nu);
    c.lcnu = (1.0 - nu) * std::log(2.0) - std::lgamma(nu);
    c.dlcnu = -std::log(2.0) - digamma_host(nu);
  }
  return c;
}

__device__ __forceinline__ double gvar(double x) { return 1.0 + 0.5 * sin(4.0 * PI * x); }

// ---- e^{-a}, a >= 0, for the covariance evaluations --------------------------
// Table-driven argument reduction (Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989):
// -a = k ln2/64 + r with k = round(-a 64/ln2), |r| <= ln2/128, so
// e^{-a} = 2^floor(k/64) 2^{(k mod 64)/64} e^r; 2^{j/64} comes from a table built
// at compile time from its Taylor series in long double, e^r - 1 from the
// Taylor polynomial of degree 5 (truncation below 4e-17 relative).  About 11
// FP64 operations; error about 1.5 ulp.  Returns 0 for a > 708 (below 1e-307).
constexpr long double MRA_LN2L = 0.693147180559945309417232121458176568L;

constexpr double exp2_frac(int j) {            // 2^(j/64)
  long double x = (long double)j / 64.0L * MRA_LN2L, term = 1.0L, sum = 1.0L;
  for (int k = 1; k < 40; ++k) {
    term *= x / (long double)k;
    sum += term;
  }
  return (double)sum;
}
#define MRA_EXP2_T8(b)                                                                                      \
  exp2_frac(b), exp2_frac(b + 1), exp2_frac(b + 2), exp2_frac(b + 3), exp2_frac(b + 4), exp2_frac(b + 5), \
      exp2_frac(b + 6), exp2_frac(b + 7)
#define MRA_EXP2_TAB                                                                                           \
  {                                                                                                           \
    MRA_EXP2_T8(0), MRA_EXP2_T8(8), MRA_EXP2_T8(16), MRA_EXP2_T8(24), MRA_EXP2_T8(32), MRA_EXP2_T8(40),         \
        MRA_EXP2_T8(48), MRA_EXP2_T8(56)                                                                      \
  }
static __device__ const double k_exp2_tab[64] = MRA_EXP2_TAB;
constexpr double k_exp2_tab_host[64] = MRA_EXP2_TAB;

constexpr double MRA_EXP_INV = (double)(64.0L / MRA_LN2L);                 // 64 / ln2
constexpr double MRA_EXP_C1 = (double)((long double)(long long)(MRA_LN2L / 64.0L * 4398046511104.0L) /
                                       4398046511104.0L);                  // ln2/64 to 36 bits: k C1 exact
constexpr double MRA_EXP_C2 = (double)(MRA_LN2L / 64.0L - (long double)MRA_EXP_C1);

__host__ __device__ inline double exp_neg_tab(double a, const double* tab) {
  if (!(a <= 708.0)) return 0.0;
  const double t = -a;
  const double magic = 6755399441055744.0;     // 1.5 2^52: adding it rounds to an integer
  const double kd0 = fma(t, MRA_EXP_INV, magic);
  long long kb;
#ifdef __CUDA_ARCH__
  kb = __double_as_longlong(kd0);
#else
  memcpy(&kb, &kd0, 8);
#endif
  const int k = (int)(unsigned)(kb & 0xFFFFFFFFll);
  const double kd = kd0 - magic;
  double r = fma(-kd, MRA_EXP_C1, t);
  r = fma(-kd, MRA_EXP_C2, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  q *= r;                                      // e^r - 1
  const int j = k & 63, m = k >> 6;            // k <= 0: m = floor(k / 64)
#ifdef __CUDA_ARCH__
  const double tj = __ldg(tab + j);
#else
  const double tj = tab[j];
#endif
  const double v = fma(tj, q, tj);
  const long long sb = (long long)(m + 1023) << 52;
  double s2;
#ifdef __CUDA_ARCH__
  s2 = __longlong_as_double(sb);
#else
  memcpy(&s2, &sb, 8);
#endif
  return v * s2;
}

__device__ __forceinline__ double exp_neg(double a) { return exp_neg_tab(a, k_exp2_tab); }

// Euclidean distance times s, sqrt through the reciprocal square root.
__device__ __forceinline__ double dist_scaled(double dx, double dy, double s) {
  const double u = fma(dx, dx, dy * dy);
  return u > 0.0 ? u * rsqrt(u) * s : 0.0;
}

// ---- Matern correlation of smoothness nu (family 2) --------------------------
// rho(h) = 2^(1-nu) / Gamma(nu) z^nu K_nu(z), z = sqrt(2 nu) h (the scaling of
// Eq. mat15, which is nu = 3/2; nu = 1/2 is the exponential), with the
// modified Bessel function of the second kind from its integral
//     K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt,
// evaluated by the trapezoidal rule, whose error falls exponentially with
// 1/step for an integrand analytic in a strip around the real axis
// (Trefethen & Weideman, "The exponentially convergent trapezoidal rule",
// SIAM Review 56, 2014): step min(0.2, 0.5/sqrt(z), 0.9/(1+nu)), nodes until
// z (cosh t - 1) - max(nu, 1 - nu) t > 40.  The same nodes give K_{nu-1}, whence
// d(z^nu K_nu)/dz = -z^nu K_{nu-1}, and dK/dnu (integrand t sinh(nu t)).  Relative error below about 1e-13 for
// nu in [0.3, 6] and z in [1e-8, 600] (checked on the host against the
// modified Bessel function of a library); sums are taken relative to e^{-z},
// so rho = c_nu exp(nu log z - z) h S0 never overflows.
struct MaternNu {
  double rho, dh, dnu;   // rho, d rho / d h, d rho / d nu (h fixed)
};

__host__ __device__ inline MaternNu matern_nu(const Cov& c, double h) {
  if (!(h > 0.0)) return MaternNu{1.0, 0.0, 0.0};
  const double nu = c.nu, z = c.snu * h;
#ifdef __CUDA_ARCH__
  const double* tab = k_exp2_tab;
  const double rz = rsqrt(z);
#else
  const double* tab = k_exp2_tab_host;
  const double rz = 1.0 / std::sqrt(z);
#endif
  const double q = fmin(fmin(0.2, 0.5 * rz), 0.9 / (1.0 + nu));
  // e^{t}, e^{nu t} and e^{(nu - 1) t} at the nodes t = k q, by recurrence
  const double e1 = exp(q), e1n = exp(nu * q), e1m = exp((nu - 1.0) * q);
  const double ie1 = 1.0 / e1, ie1n = 1.0 / e1n, ie1m = 1.0 / e1m;
  double E = 1.0, Ei = 1.0, En = 1.0, Eni = 1.0, Em = 1.0, Emi = 1.0;
  double s0 = 0.5, s2 = 0.0, s3 = 0.5;          // t = 0: weight 1/2, cosh = 1, t sinh(nu t) = 0
  for (int k = 1; k < 4096; ++k) {
    E *= e1;
    Ei *= ie1;
    En *= e1n;
    Eni *= ie1n;
    Em *= e1m;
    Emi *= ie1m;
    const double t = k * q;
    const double cm1 = 0.5 * (E + Ei) - 1.0;        // cosh t - 1
    const double ex = z * cm1;
    const double w = exp_neg_tab(ex, tab);
    s0 = fma(w, 0.5 * (En + Eni), s0);              // cosh(nu t)
    s2 = fma(w * t, 0.5 * (En - Eni), s2);          // t sinh(nu t)
    s3 = fma(w, 0.5 * (Em + Emi), s3);              // cosh((nu - 1) t)
    if (ex - fmax(nu, 1.0 - nu) * t > 40.0) break;   // (the order-(nu - 1) integrand decays at 1 - nu)
  }
  const double lz = log(z);
  const double rho = exp(c.lcnu + nu * lz - z) * q * s0;
  const double r2 = s2 / s0, r3 = s3 / s0;         // (dK_nu/dnu) / K_nu and K_{nu-1} / K_nu
  // d(z^nu K_nu(z))/dz = -z^nu K_{nu-1}(z), so d rho / d z = -rho K_{nu-1}/K_nu; d z / d h = sqrt(2 nu)
  const double dh = -rho * r3 * c.snu;
  // d log rho / d nu = d log c_nu + log z + (dK/dnu)/K + (dz/dnu) (nu/z + K'/K), dz/dnu = z / (2 nu),
  // and nu/z + K'/K = -K_{nu-1}/K
  const double dnu = rho * (c.dlcnu + lz + r2 - 0.5 * z / nu * r3);
  return MaternNu{rho, dh, dnu};
}

__device__ __forceinline__ double cov0(const Cov& c, double x1, double y1, double x2, double y2) {
  double rho;
  if (c.family == 2) {
    rho = matern_nu(c, dist_scaled(x1 - x2, y1 - y2, c.ik)).rho;
  } else if (c.family == 0) {
    rho = exp_neg(dist_scaled(x1 - x2, y1 - y2, c.ik));
  } else {
    const double a = dist_scaled(x1 - x2, y1 - y2, SQRT3 * c.ik);
    const double e = exp_neg(a);
    rho = fma(a, e, e);                        // (1 + a) e^{-a}
  }
  double v = c.sigma2 * rho;
  if (c.nonstat) v *= sqrt(gvar(x1) * gvar(x2));
  return v;
}

// ---- C0 with few FP64 operations (families 0 and 1) -------------------------
// GB300 retires about 2 FP64 FMA per clock per SM against 128 FP32 operations,
// and the emulated form's kernels evaluate n M r covariances per evaluation,
// so these form C0 from the squared scaled distance u = (s dx)^2 + (s dy)^2
// (s = 1/kappa for the exponential, sqrt(3)/kappa for Matern-1.5) and a
// variance factor sc with 8 (exponential) or 9 (Matern-1.5) FP64 operations,
// the rest on the FP32 and integer pipes:
//  * a = sqrt(u): an FP32 reciprocal square root corrected once in
//    double-float arithmetic (Dekker, "A floating-point technique for
//    extending the available precision", Numer. Math. 18, 1971), which is
//    good to about 2^-44, then one FP64 Newton step;
//  * e^{-a} = 2^{-m} 2^{-j/4096} e^{-r} with k = 4096 m + j the nearest
//    integer to a 4096/ln2 (from the double-float seed), r = a - k ln2/4096 in
//    FP64 with ln2/4096 split so that k C1 is exact (Cody & Waite), and
//    e^{-r} - 1 = -r + r^2/2 - r^3/6 + r^4/24 in double-float (|r| <= 8.5e-5:
//    truncation below 2^-70); 2^{-j/4096} from a 4096-entry table and 2^{-m}
//    folded into sc through the exponent field.
// Error within a few ulp of the exactly rounded value, plus a 2^-53 relative
// (as for any evaluation from a rounded distance); a > 708 gives 0, as
// exp_neg does.
constexpr int C0_GMAX = 16;                    // knot-grid sides whose squared offsets the kernels tabulate

constexpr long double exp2n_frac(int j, int den) {   // 2^{-j/den} by its Taylor series
  long double x = -(long double)j / (long double)den * MRA_LN2L, term = 1.0L, sum = 1.0L;
  for (int k = 1; k < 40; ++k) {
    term *= x / (long double)k;
    sum += term;
  }
  return sum;
}
struct C0Tab {
  double v[4096];
};
constexpr C0Tab make_c0_tab() {              // 2^{-j/4096} = 2^{-(j>>6)/64} 2^{-(j&63)/4096}
  C0Tab t{};
  for (int j = 0; j < 4096; ++j) t.v[j] = (double)(exp2n_frac(j >> 6, 64) * exp2n_frac(j & 63, 4096));
  return t;
}
static __device__ const C0Tab k_c0_tab = make_c0_tab();
constexpr long double MRA_C0_L = MRA_LN2L / 4096.0L;
constexpr double MRA_C0_C1 = (double)((long double)(long long)(MRA_C0_L * 8796093022208.0L) /
                                      8796093022208.0L);          // ln2/4096 to 2^-43: k C1 exact for k < 2^22
constexpr double MRA_C0_C2 = (double)(MRA_C0_L - (long double)MRA_C0_C1);
constexpr float MRA_C0_I1 = (float)(1.0L / MRA_C0_L);                // 4096/ln2 as two floats
constexpr float MRA_C0_I2 = (float)(1.0L / MRA_C0_L - (long double)MRA_C0_I1);

__host__ __device__ inline uint64_t c0_dbits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ inline double c0_bitsd(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ inline uint32_t c0_bitsf(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
__host__ __device__ inline float c0_fbits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
// Exact float -> double by bit moves (0 for zero and subnormal floats).
__host__ __device__ inline double c0_widen(float f) {
  const uint32_t u = c0_bitsf(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  return c0_bitsd(((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                  ((uint64_t)(u & 0x7FFFFFu) << 29));
}
// x = hi + lo: hi the leading 24 bits of x, lo the other 29 rounded to 24, for
// 2^-70 <= |x| < 2^127 (both 0 below).
__host__ __device__ inline void c0_split(double x, float& hi, float& lo) {
  const uint64_t b = c0_dbits(x);
  const uint32_t h = (uint32_t)(b >> 32);
  const int be = (int)((h >> 20) & 0x7FFu);
  if (be < 953) {
    hi = lo = 0.f;
    return;
  }
  const uint32_t sg = h & 0x80000000u;
  hi = c0_fbits(sg | ((uint32_t)(be - 896) << 23) | ((uint32_t)(b >> 29) & 0x7FFFFFu));
  const float rem = (float)(uint32_t)(b & 0x1FFFFFFFu) * c0_fbits((uint32_t)(be - 948) << 23);   // x 2^(be-1075)
  lo = sg ? -rem : rem;
}

// C0 (v), sc e^{-a} (e) and a = sqrt(u), from which the gradient's derivative
// pairs follow: dC0/dsigma2 = v / sigma2, dC0/dkappa = e a / kappa
// (exponential) or e a^2 / kappa (Matern-1.5).
struct C0Val {
  double v, e, a;
};

__host__ __device__ inline C0Val c0_eval(int family, double u, double sc) {
  float uh, ul;
  c0_split(u, uh, ul);
  if (!(uh >= 0x1p-60f)) {                     // zero or tiny distance: the plain evaluation
#ifdef __CUDA_ARCH__
    const double a = u > 0.0 ? sqrt(u) : 0.0;
    const double e = sc * exp_neg_tab(a, k_exp2_tab);
#else
    const double a = u > 0.0 ? std::sqrt(u) : 0.0;
    const double e = sc * exp_neg_tab(a, k_exp2_tab_host);
#endif
    return C0Val{family == 0 ? e : fma(a, e, e), e, a};
  }
  if (uh > 501264.0f) return C0Val{0.0, 0.0, 708.0};   // a > 708
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(uh);
  const double* tab = k_c0_tab.v;
#else
  const float y = 1.0f / std::sqrt(uh);
  static constexpr C0Tab tabh = make_c0_tab();
  const double* tab = tabh.v;
#endif
  // a = sqrt(u): double-float seed (ah, al), then one FP64 Newton step
  const float ah = uh * y, hy = 0.5f * y;
  const float p = ah * ah, pe = fmaf(ah, ah, -p);
  const float al = (((uh - p) - pe) + ul) * hy;
  const double a0 = c0_widen(ah) + c0_widen(al);
  const double a = fma(c0_widen(hy), fma(-a0, a0, u), a0);
  // k = nearest integer to a 4096/ln2, from the seed in double-float
  const float th = ah * MRA_C0_I1;
  const float tl = fmaf(ah, MRA_C0_I1, -th) + fmaf(ah, MRA_C0_I2, al * MRA_C0_I1);
  float kf = rintf(th);
  const float fr = (th - kf) + tl;
  kf += fr > 0.5f ? 1.0f : (fr < -0.5f ? -1.0f : 0.0f);
  const int k = (int)kf;
  const double kd = c0_widen(kf);
  double rr = fma(kd, -MRA_C0_C1, a);
  rr = fma(kd, -MRA_C0_C2, rr);
  // g = e^{-r} - 1 = -r + r^2/2 - r^3/6 + r^4/24, r = rh + rl, as gh + gl
  float rh, rl;
  c0_split(rr, rh, rl);
  const float p2 = rh * rh, e2 = fmaf(rh, rh, -p2);
  const float hp = 0.5f * p2;
  const float gh = hp - rh;                    // two-sum of -rh and hp
  const float bb = gh - hp;
  const float er = (hp - (gh - bb)) + (-rh - bb);
  const float small = fmaf(0.5f, e2, fmaf(rh, rl, -rl)) + p2 * fmaf(p2, 1.0f / 24.0f, -rh * (1.0f / 6.0f));
  const double gd = c0_widen(gh) + c0_widen(er + small);
  // sc 2^{-m} by the exponent field (sc > 0 normal), then sc e^{-a}
  const int j = k & 4095, m = k >> 12;
  const uint64_t sb = c0_dbits(sc);
  if ((int)(sb >> 52) <= m) return C0Val{0.0, 0.0, a};   // below 2^-1022
#ifdef __CUDA_ARCH__
  const double tj = __ldg(tab + j);
#else
  const double tj = tab[j];
#endif
  const double tw = tj * c0_bitsd(sb - ((uint64_t)m << 52));
  const double E = fma(tw, gd, tw);
  return C0Val{family == 0 ? E : fma(a, E, E), E, a};   // Matern-1.5: (1 + a) e^{-a}
}

__host__ __device__ inline double c0_fast(int family, double u, double sc) { return c0_eval(family, u, sc).v; }

// Variance factor of C0 at a point: sqrt(1 + 0.5 sin(4 pi x)) for the
// nonstationary variance (so that C0's factor is the product at the two
// points), else 1.
__device__ __forceinline__ double c0_vfac(const Cov& c, double x) { return c.nonstat ? sqrt(gvar(x)) : 1.0; }

// Scale s of the squared distance c0_fast takes.
__host__ __device__ inline double c0_scale(const Cov& c) { return c.family == 0 ? c.ik : SQRT3 * c.ik; }

// Whether the kernels may use c0_fast on a knot grid of gx x gy.
__host__ __device__ inline bool c0_fast_ok(const Cov& c, int gx, int gy) {
  return c.family != 2 && gx <= C0_GMAX && gy <= C0_GMAX;
}

// Binary exponent e with |x| < 2^e (-2000 for zero): the row and column
// scales of the FP64-emulation engine.
__device__ __forceinline__ int xexp_of(double x) {
  const int be = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
  return be == 0 ? -2000 : be - 1022;
}

// ---- partition and knots (Sec. 2.2) -----------------------------------------
// Every level-(m-1) region splits the same way: into an s_x x s_y grid of equal
// children, s_x = 2^hx_m, s_y = 2^hy_m (J_m = s_x s_y; the midpoint quadtree is
// hx_m = hy_m = 1), each side cut by repeated midpoint halving, half-open with
// the last cell closed.  Child digit j = c_x + s_x c_y; region i of level m
// holds its digits from the top level down, level t's in the hx_t + hy_t bits
// below those of the levels above.  hx_m and hy_m sit in bits 4m..4m+3 of two
// packed words (levels 1..12).
struct Box { double x0, x1, y0, y1; };

__host__ __device__ __forceinline__ int lvl_hx(unsigned long long hx, int m) { return (int)((hx >> (4 * m)) & 15ull); }
__host__ __device__ __forceinline__ int lvl_bits(unsigned long long hx, unsigned long long hy, int m) {
  return lvl_hx(hx, m) + lvl_hx(hy, m);
}
// bits of a level-m region id: hx_1 + hy_1 + ... + hx_m + hy_m
__host__ __device__ __forceinline__ int lvl_depth(unsigned long long hx, unsigned long long hy, int m) {
  int d = 0;
  for (int t = 1; t <= m; ++t) d += lvl_bits(hx, hy, t);
  return d;
}

__device__ __forceinline__ Box region_box(const double* bbox, unsigned long long hx, unsigned long long hy, int m,
                                          long i) {
  Box b{bbox[0], bbox[1], bbox[2], bbox[3]};
  int sh = lvl_depth(hx, hy, m);
  for (int t = 1; t <= m; ++t) {
    const int a = lvl_hx(hx, t), c = lvl_hx(hy, t);
    sh -= a + c;
    const long j = (i >> sh) & ((1L << (a + c)) - 1);
    const long cx = j & ((1L << a) - 1), cy = j >> a;
    for (int q = a - 1; q >= 0; --q) {
      const double xm = 0.5 * (b.x0 + b.x1);
      if ((cx >> q) & 1) b.x0 = xm; else b.x1 = xm;
    }
    for (int q = c - 1; q >= 0; --q) {
      const double ym = 0.5 * (b.y0 + b.y1);
      if ((cy >> q) & 1) b.y0 = ym; else b.y1 = ym;
    }
  }
  return b;
}

// Knot q = a + gx * b of a gx x gy cell-centred grid in box.
__device__ __forceinline__ void knot_xy(const Box& b, int gx, int gy, int q, double& x, double& y) {
  int a = q % gx, c = q / gx;
  x = b.x0 + ((a + 0.5) * (b.x1 - b.x0)) / gx;
  y = b.y0 + ((c + 0.5) * (b.y1 - b.y0)) / gy;
}

// ---- register-blocked tile product ------------------------------------------
// acc(i, j) += sum_k A(i, k) * B(j, k) for i < na, j < nb (both <= TILE).
// A(i, k) = A[i * sai + k * sak] and B(j, k) = B[j * sbj + k * sbk]: either
// operand may be row-major (sak = 1) or k-major (sai = 1).  Operands are staged
// k-major through shared memory in chunks of KC; the 16 x 16 thread grid gives
// every thread an RM x RM block of the TILE x TILE output (RM = TILE / 16).
template <int TILE>
struct TileAcc {
  static constexpr int RM = TILE / 16;
  double v[RM][RM];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
      for (int b = 0; b < RM; ++b) v[a][b] = 0.0;
  }
  __device__ __forceinline__ int row(int a) const { return (threadIdx.x >> 4) * RM + a; }
  __device__ __forceinline__ int col(int b) const { return (threadIdx.x & 15) * RM + b; }
};

template <int TILE>
constexpr int tile_smem_doubles() { return 2 * KC * (TILE + 2); }

template <int TILE>
__device__ __forceinline__ void stage(double* s, const double* X, long sxi, long sxk, int nx,
                                      int k0, int kn) {
  constexpr int LD = TILE + 2;
  if (sxk == 1) {          // row-major source: threads along k for coalescing
    for (int t = threadIdx.x; t < TILE * KC; t += NT) {
      int i = t / KC, k = t - i * KC;
      s[k * LD + i] = (i < nx && k < kn) ? X[i * sxi + (long)(k0 + k)] : 0.0;
    }
  } else {                 // k-major source: threads along i
    for (int t = threadIdx.x; t < TILE * KC; t += NT) {
      int k = t / TILE, i = t - k * TILE;
      s[k * LD + i] = (i < nx && k < kn) ? X[(long)(k0 + k) * sxk + i * sxi] : 0.0;
    }
  }
}

template <int TILE>
__device__ void tile_mma(TileAcc<TILE>& acc, const double* A, long sai, long sak, int na,
                         const double* B, long sbj, long sbk, int nb, int K, double* smem) {
  constexpr int LD = TILE + 2;
  constexpr int RM = TILE / 16;
  double* sA = smem;
  double* sB = smem + KC * LD;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int k0 = 0; k0 < K; k0 += KC) {
    int kn = min(KC, K - k0);
    __syncthreads();
    stage<TILE>(sA, A, sai, sak, na, k0, kn);
    stage<TILE>(sB, B, sbj, sbk, nb, k0, kn);
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kn; ++k) {
      double a[RM], b[RM];
#pragma unroll
      for (int q = 0; q < RM; ++q) {
        a[q] = sA[k * LD + ty * RM + q];
        b[q] = sB[k * LD + tx * RM + q];
      }
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) acc.v[p][q] = fma(a[p], b[q], acc.v[p][q]);
    }
  }
  __syncthreads();
}

// The same product on a TR x TC output tile (TR, TC multiples of 16): the 16 x
// 16 thread grid gives every thread an (TR / 16) x (TC / 16) block, so a tile
// of few rows (prediction points) against TC columns wastes no FMA lanes on
// empty rows.
template <int TR, int TC>
struct TileAccR {
  static constexpr int RR = TR / 16, RC = TC / 16;
  double v[RR][RC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int a = 0; a < RR; ++a)
#pragma unroll
      for (int b = 0; b < RC; ++b) v[a][b] = 0.0;
  }
  __device__ __forceinline__ int row(int a) const { return (threadIdx.x >> 4) * RR + a; }
  __device__ __forceinline__ int col(int b) const { return (threadIdx.x & 15) * RC + b; }
};

template <int TR, int TC>
__device__ void tile_mma_r(TileAccR<TR, TC>& acc, const double* A, long sai, long sak, int na, const double* B,
                           long sbj, long sbk, int nb, int K, double* smem) {
  constexpr int LDA = TR + 2, LDB = TC + 2;
  constexpr int RR = TR / 16, RC = TC / 16;
  double* sA = smem;
  double* sB = smem + KC * LDA;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int k0 = 0; k0 < K; k0 += KC) {
    int kn = min(KC, K - k0);
    __syncthreads();
    stage<TR>(sA, A, sai, sak, na, k0, kn);
    stage<TC>(sB, B, sbj, sbk, nb, k0, kn);
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kn; ++k) {
      double a[RR], b[RC];
#pragma unroll
      for (int q = 0; q < RR; ++q) a[q] = sA[k * LDA + ty * RR + q];
#pragma unroll
      for (int q = 0; q < RC; ++q) b[q] = sB[k * LDB + tx * RC + q];
#pragma unroll
      for (int p = 0; p < RR; ++p)
#pragma unroll
        for (int q = 0; q < RC; ++q) acc.v[p][q] = fma(a[p], b[q], acc.v[p][q]);
    }
  }
  __syncthreads();
}

// ---- factorisations in shared memory ----------------------------------------
// Lower Cholesky factor in place (A = L L'); the strict upper triangle is set
// to zero.  A non-positive (or NaN) pivot sets *bad and is replaced by 1 so
// the factorisation stays finite.  Returns nothing; ends with __syncthreads.
// Packed lower-triangle index t -> (i, k), k <= i, t = i (i + 1) / 2 + k.
__device__ __forceinline__ void tri_decode(int t, int& i, int& k) {
  int ii = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (ii * (ii + 1) / 2 > t) --ii;
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  i = ii;
  k = t - ii * (ii + 1) / 2;
}

__device__ inline void chol_smem(double* A, int n, int lda, int* bad) {
  // The pivot of column j (L_jj = d rsqrt(d), and rsqrt(d) to scale the
  // column; long sequences on this chip's narrow FP64 pipe) is formed by
  // thread 0 alone, right after it has
  // applied the previous column's update to A_jj (element t = 0 of the
  // trailing update is always its own), while the other threads update the
  // rest of the trailing block.
  __shared__ double piv;
  __syncthreads();
  if (threadIdx.x == 0 && n > 0) {
    const double d = A[0];
    const bool ok = d > 0.0;
    const double rs = ok ? rsqrt(d) : 1.0;
    if (!ok) *bad = 1;
    A[0] = ok ? d * rs : 1.0;
    piv = rs;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double inv = piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += NT) A[i * lda + j] *= inv;
    __syncthreads();                       // column j scaled; piv read by every thread
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * (m + 1) / 2; t += NT) {   // lower triangle of the trailing block
      int ii, kk;
      tri_decode(t, ii, kk);
      const int i = j + 1 + ii, k = j + 1 + kk;
      const double v = fma(-A[i * lda + j], A[k * lda + j], A[i * lda + k]);
      if (t == 0) {                        // A_{j+1,j+1}: the next pivot
        const bool ok = v > 0.0;
        const double rs = ok ? rsqrt(v) : 1.0;
        if (!ok) *bad = 1;
        A[i * lda + k] = ok ? v * rs : 1.0;
        piv = rs;
      } else {
        A[i * lda + k] = v;
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int i = t / n, k = t - i * n;
    if (k > i) A[i * lda + k] = 0.0;
  }
  __syncthreads();
}

// ---- block-diagonal factorisations (a group of leaves in one CTA) ---------
// The nb diagonal blocks of A start at rows seg[0] = 0 <= seg[1] <= ... <=
// seg[nb] (= the order of A).  chol_seg factorises every block in place as
// chol_smem factorises one matrix and leaves every entry outside the blocks'
// lower triangles zero; trinv_seg inverts every block's lower triangle as
// trinv_smem does (the same operations per entry, so a block's factors are
// those of the single-matrix routines).  The steps of all blocks run together,
// so the barriers are those of the largest block alone.  pv: nb doubles of
// shared memory (the blocks' pivots), tmp: seg[nb] doubles.  STK (stacked
// storage): row i holds only its block's columns, entry (i, k) of block b at
// A[i lda + k - seg[b]], lda >= the largest block.
constexpr int LGRP_MAX = 4;        // leaves of one group (the children of one parent)

__device__ __forceinline__ int seg_block(const int* seg, int nb, int i) {   // block of row i
  int b = 0;
  while (b + 1 < nb && i >= seg[b + 1]) ++b;
  return b;
}

template <bool STK = false>
__device__ inline void chol_seg(double* A, int lda, const int* seg, int nb, int* bad, double* pv) {
  __syncthreads();
  int nmax = 0;
  for (int b = 0; b < nb; ++b) nmax = max(nmax, seg[b + 1] - seg[b]);
  if (threadIdx.x < nb && seg[threadIdx.x + 1] > seg[threadIdx.x]) {
    const int s0 = seg[threadIdx.x], cs = STK ? s0 : 0;
    const double d = A[s0 * lda + s0 - cs];
    const bool ok = d > 0.0;
    const double rs = ok ? rsqrt(d) : 1.0;
    if (!ok) *bad = 1;
    A[s0 * lda + s0 - cs] = ok ? d * rs : 1.0;
    pv[threadIdx.x] = rs;
  }
  __syncthreads();
  for (int j = 0; j < nmax; ++j) {
    int tot = 0, tri = 0;
    for (int b = 0; b < nb; ++b) {
      const int m = max(0, seg[b + 1] - seg[b] - j - 1);
      tot += m;
      tri += m * (m + 1) / 2;
    }
    for (int t = threadIdx.x; t < tot; t += NT) {   // column j of every block scaled
      int b = 0, u = t;
      for (int m = max(0, seg[1] - seg[0] - j - 1); u >= m; m = max(0, seg[b + 1] - seg[b] - j - 1)) {
        u -= m;
        ++b;
      }
      const int s0 = seg[b], cs = STK ? s0 : 0;
      A[(s0 + j + 1 + u) * lda + s0 + j - cs] *= pv[b];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tri; t += NT) {   // trailing lower triangles; element 0: the next pivot
      int b = 0, u = t;
      for (int m = max(0, seg[1] - seg[0] - j - 1); u >= m * (m + 1) / 2; m = max(0, seg[b + 1] - seg[b] - j - 1)) {
        u -= m * (m + 1) / 2;
        ++b;
      }
      int ii, kk;
      tri_decode(u, ii, kk);
      const int s0 = seg[b], cs = STK ? s0 : 0, jc = s0 + j, i = jc + 1 + ii, k = jc + 1 + kk;
      const double v = fma(-A[i * lda + jc - cs], A[k * lda + jc - cs], A[i * lda + k - cs]);
      if (u == 0) {
        const bool ok = v > 0.0;
        const double rs = ok ? rsqrt(v) : 1.0;
        if (!ok) *bad = 1;
        A[i * lda + k - cs] = ok ? v * rs : 1.0;
        pv[b] = rs;
      } else {
        A[i * lda + k - cs] = v;
      }
    }
    __syncthreads();
  }
  const int n = seg[nb];
  if (STK) {                                   // (stacked: row i holds its block's columns only, lda of them)
    for (int t = threadIdx.x; t < n * lda; t += NT) {
      const int i = t / lda, k = t - i * lda;
      if (k > i - seg[seg_block(seg, nb, i)]) A[t] = 0.0;
    }
  } else {
    for (int t = threadIdx.x; t < n * n; t += NT) {
      const int i = t / n, k = t - i * n;
      if (k > i || k < seg[seg_block(seg, nb, i)]) A[i * lda + k] = 0.0;
    }
  }
  __syncthreads();
}

template <bool STK = false>
__device__ inline void trinv_seg(double* A, int lda, const int* seg, int nb, double* tmp, double* pv) {
  __syncthreads();
  int nmax = 0;
  for (int b = 0; b < nb; ++b) nmax = max(nmax, seg[b + 1] - seg[b]);
  if (threadIdx.x < nb && seg[threadIdx.x + 1] > seg[threadIdx.x]) {
    const int s0 = seg[threadIdx.x];
    pv[threadIdx.x] = 1.0 / A[s0 * lda + (STK ? 0 : s0)];
  }
  __syncthreads();
  for (int k = 0; k < nmax; ++k) {
    // phase 1, every block with k < n_b: row k scaled by 1 / L_kk (X_kk = 1 / L_kk), and
    // column k below the diagonal saved
    int tot = 0, upd = 0;
    for (int b = 0; b < nb; ++b) {
      const int nbk = seg[b + 1] - seg[b];
      if (k < nbk) {
        tot += nbk;
        upd += (nbk - k - 1) * (k + 1);
      }
    }
    for (int t = threadIdx.x; t < tot; t += NT) {
      int b = 0, u = t;
      for (int c = k < seg[1] - seg[0] ? seg[1] - seg[0] : 0; u >= c;
           c = k < seg[b + 1] - seg[b] ? seg[b + 1] - seg[b] : 0) {
        u -= c;
        ++b;
      }
      const int s0 = seg[b], cs = STK ? s0 : 0, gk = s0 + k;
      if (u <= k) A[gk * lda + s0 + u - cs] = u < k ? A[gk * lda + s0 + u - cs] * pv[b] : pv[b];
      else tmp[s0 + u] = A[(s0 + u) * lda + gk - cs];
    }
    __syncthreads();
    if (threadIdx.x < nb) {   // the next step's reciprocals (diagonal entries phase 2 does not write)
      const int s0 = seg[threadIdx.x], cs = STK ? s0 : 0;
      if (k + 1 < seg[threadIdx.x + 1] - s0) pv[threadIdx.x] = 1.0 / A[(s0 + k + 1) * lda + s0 + k + 1 - cs];
    }
    // phase 2: X_ij -= L_ik X_kj for i > k, j <= k, within every block
    const int w = k + 1;
    for (int t = threadIdx.x; t < upd; t += NT) {
      int b = 0, u = t;
      for (int c = k < seg[1] - seg[0] ? (seg[1] - seg[0] - k - 1) * w : 0; u >= c;
           c = k < seg[b + 1] - seg[b] ? (seg[b + 1] - seg[b] - k - 1) * w : 0) {
        u -= c;
        ++b;
      }
      const int s0 = seg[b], cs = STK ? s0 : 0, ii = u / w, j = u - ii * w, i = s0 + k + 1 + ii;
      const double x0 = j == k ? 0.0 : A[i * lda + s0 + j - cs];
      A[i * lda + s0 + j - cs] = fma(-tmp[i], A[(s0 + k) * lda + s0 + j - cs], x0);
    }
    __syncthreads();
  }
}

// Lower-triangular L in place -> L^{-1}, by forward substitution on the rows
// of the identity (right-looking): step k scales row k by 1 / L_kk and
// subtracts L_ik times it from every row i > k.  Each step is a rank-1 update
// over all threads, so the FP64 work is spread over every warp (the pipe of
// every SM sub-partition).  tmp: n doubles of shared scratch.
__device__ inline void trinv_smem(double* A, int n, int lda, double* tmp) {
  __shared__ double piv;
  __syncthreads();
  if (threadIdx.x == 0 && n > 0) piv = 1.0 / A[0];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // phase 1: row k of X (columns < k) scaled by 1 / L_kk, X_kk = 1 / L_kk;
    // column k of L below the diagonal saved before it is overwritten
    const double rk = piv;
    for (int t = threadIdx.x; t <= k; t += NT) A[k * lda + t] = t < k ? A[k * lda + t] * rk : rk;
    for (int i = k + 1 + threadIdx.x; i < n; i += NT) tmp[i] = A[i * lda + k];
    __syncthreads();
    if (threadIdx.x == 0 && k + 1 < n) piv = 1.0 / A[(k + 1) * lda + k + 1];   // next step's reciprocal
    // phase 2: X_ij -= L_ik X_kj for i > k, j <= k (X_ik starts from 0)
    const int w = k + 1, nr = n - k - 1;
    for (int t = threadIdx.x; t < nr * w; t += NT) {
      const int ii = t / w, j = t - ii * w, i = k + 1 + ii;
      const double x0 = j == k ? 0.0 : A[i * lda + j];
      A[i * lda + j] = fma(-tmp[i], A[k * lda + j], x0);
    }
    __syncthreads();
  }
}

// ---- reductions --------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// d C0 / d sigma2, d C0 / d kappa and (family 2) d C0 / d nu at one pair of points.
__device__ __forceinline__ void dcov0(const Cov& c, double x1, double y1, double x2, double y2, double& ds2,
                                      double& dk, double& dnu) {
  double rho, drho;   // rho(h/kappa) and kappa * d rho / d kappa (= -h rho'(h))
  dnu = 0.0;
  if (c.family == 2) {
    const double h = dist_scaled(x1 - x2, y1 - y2, c.ik);
    const MaternNu mv = matern_nu(c, h);
    rho = mv.rho;
    drho = -h * mv.dh;
    dnu = c.sigma2 * mv.dnu;
  } else if (c.family == 0) {
    const double h = dist_scaled(x1 - x2, y1 - y2, c.ik);
    rho = exp_neg(h);
    drho = rho * h;
  } else {
    const double a = dist_scaled(x1 - x2, y1 - y2, SQRT3 * c.ik);
    const double e = exp_neg(a);
    rho = fma(a, e, e);
    drho = a * a * e;
  }
  double gg = c.nonstat ? sqrt(gvar(x1) * gvar(x2)) : 1.0;
  ds2 = rho * gg;
  dk = c.sigma2 * drho * gg * c.ik;
  dnu *= gg;
}

// C0 at one pair of points (rounded exactly as cov0) and, from the same
// exponential, dcov0's two derivatives (rounded exactly as dcov0).
__device__ __forceinline__ double cov0_d(const Cov& c, double x1, double y1, double x2, double y2, double& ds2,
                                         double& dk) {
  double rho, drho;
  if (c.family == 2) {   // (the gradient keeps no derivative cache for this family: it also needs d/dnu)
    const double h = dist_scaled(x1 - x2, y1 - y2, c.ik);
    const MaternNu mv = matern_nu(c, h);
    rho = mv.rho;
    drho = -h * mv.dh;
  } else if (c.family == 0) {
    const double h = dist_scaled(x1 - x2, y1 - y2, c.ik);
    rho = exp_neg(h);
    drho = rho * h;
  } else {
    const double a = dist_scaled(x1 - x2, y1 - y2, SQRT3 * c.ik);
    const double e = exp_neg(a);
    rho = fma(a, e, e);
    drho = a * a * e;
  }
  const double gg = c.nonstat ? sqrt(gvar(x1) * gvar(x2)) : 1.0;
  ds2 = rho * gg;
  dk = c.sigma2 * drho * gg * c.ik;
  double v = c.sigma2 * rho;
  if (c.nonstat) v *= gg;
  return v;
}

// Sum over the CTA; every thread gets the result.  red: 32 doubles of shared.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Lower-tile index of block (k, l), k >= l, in a packed block-lower store.
__host__ __device__ __forceinline__ int tri_index(int k, int l) { return k * (k + 1) / 2 + l; }

}  // namespace mra
