// Device-side building blocks of the MCBTE GB300 library: Philox4x32-10,
// random-word maps, per-run geometry records, ray / face / pore hits and
// direction sampling.  Everything here is templated on the tracing real
// type R (double for the FP64 path, float for the FP32 path).
//
// Internal units: length nm, time ps, velocity nm/ps.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mcbte.h"

namespace mcbte {

constexpr int kMaxGeoms = 128;
constexpr int kMaxSources = 8;
constexpr int kMaxDirs = 16;
constexpr int kMaxPeriods = 65;
constexpr int kMaxInner = MCBTE_MAX_INNER;

// Specular threshold of a reflection probability p on a 32-bit word:
// specular iff word < floor(p 2^32) (p = 1: always).
__host__ __device__ __forceinline__ uint64_t spec_threshold(double p) {
  if (p <= 0.0) return 0ull;
  if (p >= 1.0) return 1ull << 32;
  return (uint64_t)(p * 4294967296.0);
}

// ------------------------------------------------------------------ per-run records
// Geometry as the tracer sees it, derived on the device by the setup kernel
// from the caller's SI descriptor (lengths in nm, specularities as 32-bit
// integer thresholds, isothermal faces and sources resolved).
struct alignas(128) GeoRun {
  // What the FP32 event step reads at every event, together in the record's
  // first 128 bytes (one L1 line: a batch of many geometries keeps every
  // geometry's line cached); the rest is read at emission or by the FP64 path.
  float Lf[3];
  float cxf, cyf, r2f;
  int pore;
  int n_inner;
  int fbin;                    // bit f: face f takes the per-bin specularity
  int sbin;                    // bit k: wall k takes the per-bin specularity
  int unfold;                  // bit a: axis a is periodic and the box holds no pore or wall
  int type[6];
  uint64_t pthr[6];
  uint64_t pthr_pore;
  double L[3];
  double cx, cy, r2;
  // internal walls (Sec. 4.2), nm, oriented as given; normal into the solid
  double sx1[kMaxInner], sy1[kMaxInner], sx2[kMaxInner], sy2[kMaxInner], snx[kMaxInner], sny[kMaxInner];
  float sx1f[kMaxInner], sy1f[kMaxInner], sx2f[kMaxInner], sy2f[kMaxInner], snxf[kMaxInner], snyf[kMaxInner];
  uint64_t sthr[kMaxInner];
  int n_src;
  int src_kind[kMaxSources];   // 0 isothermal face, 1 body (control gradient), 2 initial Gaussian
  int src_face[kMaxSources];
  uint64_t src_thr[kMaxSources];
  double face_sign[6];         // sign of T_b - T_eq of isothermal faces
  int grad_axis;
  double grad_sign;
  int grad_general;            // gradient with several components: Lambertian about -+grad T
  double gframe[2][9];         // frames {n, b1, b2} about -grad T/|grad T| ([0]) and +grad T/|grad T| ([1])
  float gframef[2][9];
  double gauss_c[3];
  double gauss_sigma;
  double gauss_sign;
  double p_pore;
  double E_tot;                // W (steady) or J (transient)
  double V_solid;              // m^3
  double V_box;                // m^3
  double kappa_grad;           // K/m that defines kappa along the tally axis
  uint64_t n;                  // particles of this geometry in this call
  uint64_t offset;             // first flattened particle index
  uint64_t pid0;               // index of this call's first particle within the geometry's run
  uint64_t n_norm;             // particles of the geometry's whole run (E_eff = E_tot / n_norm)
};
static_assert(offsetof(GeoRun, pthr_pore) + sizeof(uint64_t) <= 128, "FP32 per-event fields within one line");

// Material as the tracer sees it (device pointers).
struct MatView {
  int n;
  const uint4* rec_emit;    // alias records ~ C v   {thr_lo, thr_hi, alias, 0}
  const uint4* rec_init;    // alias records ~ C
  const uint4* rec_relax;   // alias records ~ C / tau
  const float4* binf;       // {v (nm/ps), 1/v (ps/nm), Lambda (nm), Lambda_2 (nm, +inf: none)}
  const double* v_d;        // nm/ps
  const double* inv_v_d;    // ps/nm
  const double* lam_d;      // nm
  const double* pi;         // relaxation pmf (C/tau) / sum(C/tau)
  const double* sums;       // [3] sum C, sum C v, sum C / tau  (SI)
  const double* lam2_d;     // nm, two-phonon mean free path v tau_imp (+inf: none)
  int imp;                  // a two-phonon clock is present (Sec. 3.3)
  const uint64_t* spec_thr; // per-bin specular thresholds floor(d(omega) 2^32), or null
};

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64 products
// with multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key schedule
// 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ------------------------------------------------------------------ FP64 elementary functions
// Fixed-order series (no library transcendental), so the FP64 tracer is a
// deterministic function of its random words on any IEEE-754 double
// arithmetic without fused multiply-add (this translation unit is built
// with --fmad=false).
//
// ln x: x = m 2^e, m folded into [sqrt(2)/2, sqrt(2)], ln x = e ln 2 +
// 2 atanh((m-1)/(m+1)); atanh by its Taylor series through z^25
// (Abramowitz & Stegun 4.1.27), Horner from the highest coefficient.
__device__ __forceinline__ double series_log(double x) {
  const long long bits = __double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7ffll) - 1023;
  double m = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    ex = ex + 1;
  }
  const double z = (m - 1.0) / (m + 1.0);
  const double z2 = z * z;
  // 1/(2k+1) for k = 12 down to 1
  const double inv_odd[12] = {0.04, 0.043478260869565216, 0.047619047619047616, 0.05263157894736842,
                              0.058823529411764705, 0.06666666666666667, 0.07692307692307693, 0.09090909090909091,
                              0.1111111111111111, 0.14285714285714285, 0.2, 0.3333333333333333};
  double p = inv_odd[0];
#pragma unroll
  for (int k = 1; k < 12; ++k) p = inv_odd[k] + z2 * p;
  const double lm = 2.0 * (z + z * (z2 * p));
  return (double)ex * 0.6931471805599453 + lm;
}

// cos(2 pi r), sin(2 pi r), r in [0, 1): octant reduction to theta in
// [0, pi/4], Taylor polynomials of sin (to theta^15) and cos (to theta^16)
// by Horner from the highest coefficient, then the octant symmetries.
__device__ __forceinline__ void series_sincos2pi(double r, double* sn, double* cs) {
  const double t = r * 8.0;
  const int oct = (int)t;
  double f = t - (double)oct;
  if (oct & 1) f = 1.0 - f;
  const double th = f * 0.7853981633974483;
  const double t2 = th * th;
  const double sc[8] = {-7.647163731819816e-13, 1.6059043836821613e-10, -2.505210838544172e-08,
                        2.7557319223985893e-06, -0.0001984126984126984, 0.008333333333333333,
                        -0.16666666666666666, 1.0};
  const double cc[9] = {4.779477332387385e-14, -1.1470745597729725e-11, 2.08767569878681e-09,
                        -2.755731922398589e-07, 2.48015873015873e-05, -0.001388888888888889,
                        0.041666666666666664, -0.5, 1.0};
  double ps = sc[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) ps = sc[k] + t2 * ps;
  double pc = cc[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) pc = cc[k] + t2 * pc;
  const double S = th * ps;
  const double C = pc;
  switch (oct & 7) {
    case 0: *cs = C; *sn = S; break;
    case 1: *cs = S; *sn = C; break;
    case 2: *cs = -S; *sn = C; break;
    case 3: *cs = -C; *sn = S; break;
    case 4: *cs = -C; *sn = -S; break;
    case 5: *cs = -S; *sn = -C; break;
    case 6: *cs = S; *sn = -C; break;
    default: *cs = C; *sn = -S; break;
  }
}

// ------------------------------------------------------------------ real maps
template <typename R> struct Num;

template <> struct Num<double> {
  static __device__ __forceinline__ double oc(uint32_t w) { return ((double)w + 1.0) * 2.3283064365386963e-10; }
  static __device__ __forceinline__ double co(uint32_t w) { return (double)w * 2.3283064365386963e-10; }
  static __device__ __forceinline__ double mid(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }
  static __device__ __forceinline__ double oc53(uint32_t lo, uint32_t hi) {
    const uint64_t m = ((uint64_t)hi << 21) ^ (uint64_t)(lo >> 11);
    return ((double)m + 1.0) * 1.1102230246251565e-16;
  }
  static __device__ __forceinline__ double log_(double x) { return series_log(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ void sincos2pi(double r, double* s, double* c) { series_sincos2pi(r, s, c); }
  static __device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double big() { return 1.0e300; }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

template <> struct Num<float> {
  static __device__ __forceinline__ float oc(uint32_t w) { return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f; }
  static __device__ __forceinline__ float co(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-8f; }
  static __device__ __forceinline__ float mid(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }
  static __device__ __forceinline__ float oc53(uint32_t lo, uint32_t hi) {
    (void)lo;
    return (float)((hi >> 8) + 1u) * 5.9604644775390625e-8f;
  }
  static __device__ __forceinline__ float log_(float x) { return __logf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ void sincos2pi(float r, float* s, float* c) {
    __sincosf(6.28318530717958647f * r, s, c);
  }
  static __device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
  // distances for the first hit: the 2-ulp hardware quotient (the particle
  // is set onto the face it hits, so the quotient's last bits move nothing)
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float big() { return 3.0e38f; }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

// Alias draw: column = floor(w * n / 2^32) (exact), keep the column iff the
// 64-bit word (hi:lo) is below its threshold, else take its alias.
__device__ __forceinline__ int alias_draw(const uint4* rec, int n, uint32_t wcol, uint32_t lo, uint32_t hi) {
  const int col = (int)(((uint64_t)wcol * (uint64_t)n) >> 32);
  const uint4 a = rec[col];
  const uint64_t thr = ((uint64_t)a.y << 32) | (uint64_t)a.x;
  const uint64_t r = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (r < thr) ? col : (int)a.z;
}

// Face index (paper ID - 1) -> axis and side.
__device__ __forceinline__ int face_axis(int f) { return (f == 1 || f == 3) ? 0 : ((f == 0 || f == 2) ? 1 : 2); }
__device__ __forceinline__ int face_is_max(int f) { return (f == 1 || f == 2 || f == 5) ? 1 : 0; }
__device__ __forceinline__ int axis_min_face(int a) { return a == 0 ? 3 : (a == 1 ? 0 : 4); }
__device__ __forceinline__ int axis_max_face(int a) { return a == 0 ? 1 : (a == 1 ? 2 : 5); }

template <typename R> __device__ __forceinline__ R geo_L(const GeoRun& g, int a);
template <> __device__ __forceinline__ double geo_L<double>(const GeoRun& g, int a) { return g.L[a]; }
template <> __device__ __forceinline__ float geo_L<float>(const GeoRun& g, int a) { return g.Lf[a]; }

// Component a of a 3-vector, and assignment to it, by selects: a runtime
// index into a register array would force the array into local memory.
template <typename R>
__device__ __forceinline__ R sel3(const R v[3], int a) {
  return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]);
}
template <typename R>
__device__ __forceinline__ void put3(R v[3], int a, R val) {
  v[0] = a == 0 ? val : v[0];
  v[1] = a == 1 ? val : v[1];
  v[2] = a == 2 ? val : v[2];
}
// v[a] = A, v[a+1] = B, v[a+2] = C (indices cyclic).
template <typename R>
__device__ __forceinline__ void put3_cyclic(R v[3], int a, R A, R B, R C) {
  v[0] = a == 0 ? A : (a == 1 ? C : B);
  v[1] = a == 0 ? B : (a == 1 ? A : C);
  v[2] = a == 0 ? C : (a == 1 ? B : A);
}

// Direction with polar cosine mu about sgn * axis a; axes a+1, a+2 (cyclic)
// take s cos(phi), s sin(phi), phi = 2 pi co(wphi).
template <typename R>
__device__ __forceinline__ void dir_about_axis(R u[3], int a, R sgn, R mu, uint32_t wphi) {
  const R s = Num<R>::sqrt_(Num<R>::fmax_(R(0), R(1) - mu * mu));
  R sn, cs;
  Num<R>::sincos2pi(Num<R>::co(wphi), &sn, &cs);
  put3_cyclic<R>(u, a, sgn * mu, s * cs, s * sn);
}

// Orthonormal frame {n, b1, b2} of n = sgn gv (gv a unit vector) by the
// branchless construction of Duff et al., "Building an Orthonormal Basis,
// Revisited" (JCGT 2017); f = {n, b1, b2} (9 values).
__host__ __device__ __forceinline__ void frame_about(const double gv[3], double sgn, double f[9]) {
  const double n0 = sgn * gv[0], n1 = sgn * gv[1], n2 = sgn * gv[2];
  const double sg = n2 >= 0.0 ? 1.0 : -1.0;
  const double a = -1.0 / (sg + n2);
  const double b = (n0 * n1) * a;
  f[0] = n0; f[1] = n1; f[2] = n2;
  f[3] = 1.0 + ((sg * n0) * n0) * a; f[4] = sg * b; f[5] = -sg * n0;
  f[6] = b; f[7] = sg + (n1 * n1) * a; f[8] = -n1;
}

// Direction with polar cosine mu about the frame's n:
// u = mu n + s cos(phi) b1 + s sin(phi) b2, phi = 2 pi co(wphi).
template <typename R>
__device__ __forceinline__ void dir_about_frame(R u[3], const R* f, R mu, uint32_t wphi) {
  const R s = Num<R>::sqrt_(Num<R>::fmax_(R(0), R(1) - mu * mu));
  R sn, cs;
  Num<R>::sincos2pi(Num<R>::co(wphi), &sn, &cs);
  const R sc = s * cs, ss = s * sn;
  u[0] = (mu * f[0] + sc * f[3]) + ss * f[6];
  u[1] = (mu * f[1] + sc * f[4]) + ss * f[7];
  u[2] = (mu * f[2] + sc * f[5]) + ss * f[8];
}

// The hardware's approximate square root (PTX sqrt.approx, a few ulp): the
// FP32 pore hit's root, where a correctly rounded root's longer instruction
// sequence sat on a lone particle's dependent chain.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP32 box faces and pore cylinder of a geometry record (GeoRun, or the
// register copy GeoLean with the same member names): the three face
// distances without branches (the quotients are independent, so their
// latencies overlap), then their minimum and the lowest paper face ID among
// the axes that reach it (the same result as scanning the axes with "nearer,
// or as near with a lower ID", with a short dependent chain: a lone
// particle's event waits on it); then the pore by the same test and root
// with selects instead of branches.  One function for both records, so both
// compute the same bits.
//
// Axes in the mask `skip` (unfolded periodic axes) take no part: the flight
// runs through their faces.
template <class Geo>
__device__ __forceinline__ void hit_box_pore_f32(const Geo& g, const float x[3], const float u[3], float* dist,
                                                 int* face, unsigned skip = 0u) {
  float c[3];
  int fa[3];
  bool ok[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float ua = u[a];
    const bool up = ua > 0.0f;
    const float d0 = Num<float>::div((up ? g.Lf[a] : 0.0f) - x[a], ua);
    ok[a] = ua != 0.0f && ((skip >> a) & 1u) == 0u;
    c[a] = ok[a] ? (d0 < 0.0f ? 0.0f : d0) : Num<float>::big();
    fa[a] = up ? axis_max_face(a) : axis_min_face(a);
  }
  float best = fminf(fminf(c[0], c[1]), c[2]);
  const int f0 = (ok[0] && c[0] == best) ? fa[0] : 7;
  const int f1 = (ok[1] && c[1] == best) ? fa[1] : 7;
  const int f2 = (ok[2] && c[2] == best) ? fa[2] : 7;
  int bf = min(min(f0, f1), f2);
  if (g.pore) {
    const float dx = x[0] - g.cxf, dy = x[1] - g.cyf;
    const float a = u[0] * u[0] + u[1] * u[1];
    const float b = dx * u[0] + dy * u[1];
    const float cc = (dx * dx + dy * dy) - g.r2f;
    const float disc = b * b - a * cc;
    const bool hit = a > 0.0f && b < 0.0f && disc >= 0.0f;
    const float d0 = Num<float>::div(cc, sqrt_approx(Num<float>::fmax_(disc, 0.0f)) - b);
    const float d = d0 < 0.0f ? 0.0f : d0;
    const bool take = hit && d < best;
    best = take ? d : best;
    bf = take ? 6 : bf;
  }
  *dist = best;
  *face = bf;
}

// The unfolded periodic axes (bits of um) folded back into [0, L) after a
// flight that ran through their faces; returns the faces crossed, each of
// them the event (a translation to the opposite face) a flight stopped at
// every face would have counted.
__device__ __forceinline__ uint32_t fold_periodic(float x[3], const float L[3], unsigned um) {
  uint32_t n = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (((um >> a) & 1u) == 0u) continue;
    const float La = L[a];
    if (x[a] >= 0.0f && x[a] < La) continue;   // no face crossed on this axis
    float k = floorf(__fdividef(x[a], La));
    float r = fmaf(-k, La, x[a]);
    // the quotient's rounding can leave r just outside [0, L)
    if (r < 0.0f) {
      r += La;
      k -= 1.0f;
    }
    if (r >= La) {
      r -= La;
      k += 1.0f;
    }
    x[a] = r;
    n += (uint32_t)fabsf(k);
  }
  return n;
}

// The FP32 event step's geometry in registers (the tail kernel's particles):
// the box, the pore, the face types packed two bits per face.
struct GeoLean {
  float Lf[3];
  float cxf, cyf, r2f;
  int pore;
  unsigned tmask;   // bits 2f..2f+1: MCBTE_FACE_* type of face f

  __device__ __forceinline__ void load(const GeoRun& g) {
#pragma unroll
    for (int a = 0; a < 3; ++a) Lf[a] = g.Lf[a];
    cxf = g.cxf;
    cyf = g.cyf;
    r2f = g.r2f;
    pore = g.pore;
    tmask = 0u;
#pragma unroll
    for (int f = 0; f < 6; ++f) tmask |= ((unsigned)g.type[f] & 3u) << (2 * f);
  }
  __device__ __forceinline__ int type(int f) const { return (int)((tmask >> (2 * f)) & 3u); }
  __device__ __forceinline__ float L(int a) const { return a == 0 ? Lf[0] : (a == 1 ? Lf[1] : Lf[2]); }
};

// First boundary along the ray (faces in the direction of travel, then the
// pore cylinder); ties go to the lowest paper boundary ID.
template <typename R, bool EXT = true>
__device__ __forceinline__ void first_hit(const GeoRun& g, const R x[3], const R u[3], R* dist, int* face) {
  R best = Num<R>::big();
  int bf = 7;
  if constexpr (sizeof(R) == 4) {
    hit_box_pore_f32(g, x, u, &best, &bf);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R d;
      int f;
      const R La = geo_L<R>(g, a);
      if (u[a] > R(0)) { d = Num<R>::div(La - x[a], u[a]); f = axis_max_face(a); }
      else if (u[a] < R(0)) { d = Num<R>::div(R(0) - x[a], u[a]); f = axis_min_face(a); }
      else continue;
      if (d < R(0)) d = R(0);
      if (d < best || (d == best && f < bf)) { best = d; bf = f; }
    }
    if (g.pore) {
      const R cx = (R)g.cx;
      const R cy = (R)g.cy;
      const R r2 = (R)g.r2;
      const R dx = x[0] - cx, dy = x[1] - cy;
      const R a = u[0] * u[0] + u[1] * u[1];
      const R b = dx * u[0] + dy * u[1];
      if (a > R(0) && b < R(0)) {
        const R c = (dx * dx + dy * dy) - r2;
        const R disc = b * b - a * c;
        if (disc >= R(0)) {
          R d = c / (Num<R>::sqrt_(disc) - b);
          if (d < R(0)) d = R(0);
          if (d < best) { best = d; bf = 6; }
        }
      }
    }
  }
  // internal walls (faces 7, 8, ...), met only from their solid side; a
  // particle behind a wall's line by more than rounding is beyond the hole
  const R tol = sizeof(R) == 8 ? R(1e-9) : R(1e-4);
  for (int k = 0; k < (EXT ? g.n_inner : 0); ++k) {
    const R nx = sizeof(R) == 8 ? (R)g.snx[k] : (R)g.snxf[k];
    const R ny = sizeof(R) == 8 ? (R)g.sny[k] : (R)g.snyf[k];
    const R un = u[0] * nx + u[1] * ny;
    const R x1 = sizeof(R) == 8 ? (R)g.sx1[k] : (R)g.sx1f[k];
    const R y1 = sizeof(R) == 8 ? (R)g.sy1[k] : (R)g.sy1f[k];
    const R dn = (x[0] - x1) * nx + (x[1] - y1) * ny;
    if constexpr (sizeof(R) == 4) {
      // FP32: every wall's candidate computed, the valid nearest selected
      const R d0 = Num<R>::div(dn, -un);
      const R d = d0 < R(0) ? R(0) : d0;
      const R tx = g.sx2f[k] - x1;
      const R ty = g.sy2f[k] - y1;
      const R hs = ((x[0] + d * u[0]) - x1) * tx + ((x[1] + d * u[1]) - y1) * ty;
      const bool take = un < R(0) && !(dn < -tol) && !(hs < R(0) || hs > tx * tx + ty * ty) && d < best;
      best = take ? d : best;
      bf = take ? 7 + k : bf;
      continue;
    }
    if (!(un < R(0))) continue;
    if (dn < -tol) continue;
    R d = dn / (-un);
    if (d < R(0)) d = R(0);
    const R tx = (sizeof(R) == 8 ? (R)g.sx2[k] : (R)g.sx2f[k]) - x1;
    const R ty = (sizeof(R) == 8 ? (R)g.sy2[k] : (R)g.sy2f[k]) - y1;
    const R hs = ((x[0] + d * u[0]) - x1) * tx + ((x[1] + d * u[1]) - y1) * ty;
    if (hs < R(0) || hs > tx * tx + ty * ty) continue;
    if (d < best) { best = d; bf = 7 + k; }
  }
  *dist = best;
  *face = bf;
}

// Inside a hole bounded by the internal walls: even-odd count of the walls
// crossed by the ray from (x, y) towards +x.
template <typename R>
__device__ __forceinline__ bool in_hole(const GeoRun& g, R x, R y) {
  bool c = false;
  for (int k = 0; k < g.n_inner; ++k) {
    const R y1 = sizeof(R) == 8 ? (R)g.sy1[k] : (R)g.sy1f[k];
    const R y2 = sizeof(R) == 8 ? (R)g.sy2[k] : (R)g.sy2f[k];
    if ((y1 > y) != (y2 > y)) {
      const R x1 = sizeof(R) == 8 ? (R)g.sx1[k] : (R)g.sx1f[k];
      const R x2 = sizeof(R) == 8 ? (R)g.sx2[k] : (R)g.sx2f[k];
      const R xc = x1 + ((y - y1) * (x2 - x1)) / (y2 - y1);
      if (x < xc) c = !c;
    }
  }
  return c;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace mcbte
