// common.cuh -- arithmetic types shared by the library's kernels.
//
// Three arithmetics run the convolution path:
//   double : native FP64 (GB300 runs it at 1/64 of the FP32 rate);
//   float  : plain FP32;
//   df     : "double-float": a value is the unevaluated sum hi + lo of two floats with
//            |lo| <= ulp(hi)/2.  Sums use Knuth's TwoSum and products Dekker/Kahan's TwoProd through
//            fmaf, so every elementary operation is error-free up to the final renormalisation
//            (about 44-48 significant bits).  All float operations go through __f*_rn intrinsics so
//            the compiler never contracts or reorders them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LGF_HD __host__ __device__ __forceinline__
#define LGF_D __device__ __forceinline__

struct df {
  float hi, lo;
};

LGF_D df df_make(double v) {
  float h = __double2float_rn(v);
  float l = __double2float_rn(v - (double)h);
  return {h, l};
}
LGF_D double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

LGF_D df df_add(df a, df b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float hi = __fadd_rn(s, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, s));
  return {hi, lo};
}
LGF_D df df_neg(df a) { return {-a.hi, -a.lo}; }
LGF_D df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
LGF_D df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float hi = __fadd_rn(p, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, p));
  return {hi, lo};
}
LGF_D df df_scale2(df a, float s) {  // exact when s is a power of two
  return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
}

LGF_D df operator+(df a, df b) { return df_add(a, b); }
LGF_D df operator-(df a, df b) { return df_sub(a, b); }
LGF_D df operator*(df a, df b) { return df_mul(a, b); }
LGF_D df operator-(df a) { return df_neg(a); }

// ------------------------------------------------------------------ scalar traits
template <class R>
struct RT;
template <>
struct RT<double> {
  LGF_D static double from(double v) { return v; }
  LGF_D static double from(float v) { return (double)v; }
  LGF_D static double to_d(double v) { return v; }
  LGF_D static float to_f(double v) { return (float)v; }
  LGF_D static double zero() { return 0.0; }
  LGF_D static double half(double v) { return 0.5 * v; }
  LGF_D static double scale(double v, double s) { return v * s; }
};
template <>
struct RT<float> {
  LGF_D static float from(double v) { return (float)v; }
  LGF_D static float from(float v) { return v; }
  LGF_D static double to_d(float v) { return (double)v; }
  LGF_D static float to_f(float v) { return v; }
  LGF_D static float zero() { return 0.0f; }
  LGF_D static float half(float v) { return 0.5f * v; }
  LGF_D static float scale(float v, double s) { return v * (float)s; }
};
template <>
struct RT<df> {
  LGF_D static df from(double v) { return df_make(v); }
  LGF_D static df from(float v) { return {v, 0.0f}; }
  LGF_D static double to_d(df v) { return df_to_double(v); }
  LGF_D static float to_f(df v) { return __fadd_rn(v.hi, v.lo); }
  LGF_D static df zero() { return {0.0f, 0.0f}; }
  LGF_D static df half(df v) { return df_scale2(v, 0.5f); }
  LGF_D static df scale(df v, double s) { return df_mul(v, df_make(s)); }
};

// ------------------------------------------------------------------ complex
// Aligned to its size so that a complex value moves as one 8- or 16-byte access (every array of cx is
// allocated by cudaMalloc or declared as cx, so element addresses keep this alignment).
template <class R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};
template <class R>
LGF_D cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
LGF_D cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
LGF_D cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
LGF_D cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <class R>
LGF_D cx<R> cx_zero() { return {RT<R>::zero(), RT<R>::zero()}; }

// ------------------------------------------------------------------ fused complex kernels
// cadd / csub / cmul / cmac: the complex sum, difference, product and multiply-add.  For double and
// float they are plain (contracted) arithmetic; for double-float they are fused error-free forms:
//   cmul: each real part is a two-term dot product: both hi*hi products by TwoProd, the four cross
//         products folded into one correction, one TwoSum, one renormalisation (19 instructions);
//   cmac: the same with the accumulator: two TwoSums, one renormalisation (27 instructions per part);
//   cadd/csub: TwoSum of the hi parts plus the lo parts, left unnormalised ("lazy"): callers
//         renormalise with cnorm before a value is stored (8 instructions per part instead of 11).
template <class R>
LGF_D cx<R> cadd(cx<R> a, cx<R> b) { return a + b; }
template <class R>
LGF_D cx<R> csub(cx<R> a, cx<R> b) { return a - b; }
template <class R>
LGF_D cx<R> cmul(cx<R> a, cx<R> b) { return a * b; }
template <class R>
LGF_D cx<R> cnorm(cx<R> a) { return a; }
LGF_D cx<double> cmac(cx<double> acc, cx<double> a, cx<double> b) {
  return {fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
}
LGF_D cx<float> cmac(cx<float> acc, cx<float> a, cx<float> b) {
  return {fmaf(a.re, b.re, fmaf(-a.im, b.im, acc.re)), fmaf(a.re, b.im, fmaf(a.im, b.re, acc.im))};
}

LGF_D df df_add_lazy(df a, df b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
LGF_D df df_sub_lazy(df a, df b) { return df_add_lazy(a, df{-b.hi, -b.lo}); }
LGF_D df df_renorm(df a) {
  float hi = __fadd_rn(a.hi, a.lo);
  return {hi, __fsub_rn(a.lo, __fsub_rn(hi, a.hi))};
}
// a*b + sgn * c*d with error-free products (sgn = +1 or -1)
LGF_D df df_dot2(df a, df b, df c, df d, float sgn) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(sgn * c.hi, d.hi);
  const float e2 = __fmaf_rn(sgn * c.hi, d.hi, -p2);
  float x = __fmaf_rn(a.lo, b.hi, e1);
  x = __fmaf_rn(a.hi, b.lo, x);
  x = __fmaf_rn(sgn * c.lo, d.hi, x);
  x = __fmaf_rn(sgn * c.hi, d.lo, __fadd_rn(x, e2));
  const float s = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  return df_renorm(df{s, __fadd_rn(t, x)});
}
// acc + a*b + sgn * c*d
LGF_D df df_dot2_acc(df acc, df a, df b, df c, df d, float sgn) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(sgn * c.hi, d.hi);
  const float e2 = __fmaf_rn(sgn * c.hi, d.hi, -p2);
  float x = __fmaf_rn(a.lo, b.hi, e1);
  x = __fmaf_rn(a.hi, b.lo, x);
  x = __fmaf_rn(sgn * c.lo, d.hi, x);
  x = __fmaf_rn(sgn * c.hi, d.lo, __fadd_rn(x, e2));
  float s = __fadd_rn(acc.hi, p1);
  float bb = __fsub_rn(s, acc.hi);
  const float t1 = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p1, bb));
  const float s2 = __fadd_rn(s, p2);
  bb = __fsub_rn(s2, s);
  const float t2 = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(p2, bb));
  const float lo = __fadd_rn(__fadd_rn(acc.lo, x), __fadd_rn(t1, t2));
  return df_renorm(df{s2, lo});
}
// acc + a*b + sgn * c*d without the final renormalisation (accumulators of a few terms)
LGF_D df df_dot2_acc_lazy(df acc, df a, df b, df c, df d, float sgn) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(sgn * c.hi, d.hi);
  const float e2 = __fmaf_rn(sgn * c.hi, d.hi, -p2);
  float x = __fmaf_rn(a.lo, b.hi, e1);
  x = __fmaf_rn(a.hi, b.lo, x);
  x = __fmaf_rn(sgn * c.lo, d.hi, x);
  x = __fmaf_rn(sgn * c.hi, d.lo, __fadd_rn(x, e2));
  float s = __fadd_rn(acc.hi, p1);
  float bb = __fsub_rn(s, acc.hi);
  const float t1 = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p1, bb));
  const float s2 = __fadd_rn(s, p2);
  bb = __fsub_rn(s2, s);
  const float t2 = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(p2, bb));
  return df{s2, __fadd_rn(__fadd_rn(acc.lo, x), __fadd_rn(t1, t2))};
}
template <>
LGF_D cx<df> cadd<df>(cx<df> a, cx<df> b) { return {df_add_lazy(a.re, b.re), df_add_lazy(a.im, b.im)}; }
template <>
LGF_D cx<df> csub<df>(cx<df> a, cx<df> b) { return {df_sub_lazy(a.re, b.re), df_sub_lazy(a.im, b.im)}; }
template <>
LGF_D cx<df> cmul<df>(cx<df> a, cx<df> b) {
  return {df_dot2(a.re, b.re, a.im, b.im, -1.0f), df_dot2(a.re, b.im, a.im, b.re, 1.0f)};
}
template <>
LGF_D cx<df> cnorm<df>(cx<df> a) { return {df_renorm(a.re), df_renorm(a.im)}; }
LGF_D cx<df> cmac(cx<df> acc, cx<df> a, cx<df> b) {
  return {df_dot2_acc(acc.re, a.re, b.re, a.im, b.im, -1.0f), df_dot2_acc(acc.im, a.re, b.im, a.im, b.re, 1.0f)};
}
// multiply-add leaving a double-float accumulator unnormalised (callers apply cnorm at the end)
LGF_D cx<double> cmac_lazy(cx<double> acc, cx<double> a, cx<double> b) { return cmac(acc, a, b); }
LGF_D cx<float> cmac_lazy(cx<float> acc, cx<float> a, cx<float> b) { return cmac(acc, a, b); }
LGF_D cx<df> cmac_lazy(cx<df> acc, cx<df> a, cx<df> b) {
  return {df_dot2_acc_lazy(acc.re, a.re, b.re, a.im, b.im, -1.0f),
          df_dot2_acc_lazy(acc.im, a.re, b.im, a.im, b.re, 1.0f)};
}

// Real-coefficient accumulations (block-index DFTs by conjugate pairs): acc + a b and acc + a b + sgn c d.
LGF_D double rfma(double acc, double a, double b) { return fma(a, b, acc); }
LGF_D float rfma(float acc, float a, float b) { return fmaf(a, b, acc); }
LGF_D df rfma(df acc, df a, df b) {  // unnormalised (callers renormalise at the end)
  const float p = __fmul_rn(a.hi, b.hi);
  float x = __fmaf_rn(a.hi, b.hi, -p);
  x = __fmaf_rn(a.lo, b.hi, x);
  x = __fmaf_rn(a.hi, b.lo, x);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return df{s, __fadd_rn(__fadd_rn(acc.lo, x), t)};
}
LGF_D double rdot2(double acc, double a, double b, double c, double d, float sgn) {
  return fma(a, b, fma((double)sgn * c, d, acc));
}
LGF_D float rdot2(float acc, float a, float b, float c, float d, float sgn) { return fmaf(a, b, fmaf(sgn * c, d, acc)); }
LGF_D df rdot2(df acc, df a, df b, df c, df d, float sgn) { return df_dot2_acc_lazy(acc, a, b, c, d, sgn); }
// x w for a float w of few significant bits (an interpolation weight): the product error is kept
// (TwoProd on the high part), the result left unnormalised
LGF_D double rscale(double x, float w) { return x * (double)w; }
LGF_D float rscale(float x, float w) { return x * w; }
LGF_D df rscale(df x, float w) {
  const float p = __fmul_rn(x.hi, w);
  return {p, __fmaf_rn(x.lo, w, __fmaf_rn(x.hi, w, -p))};
}
LGF_D double radd(double a, double b) { return a + b; }
LGF_D float radd(float a, float b) { return a + b; }
LGF_D df radd(df a, df b) { return df_add_lazy(a, b); }
template <class R>
LGF_D R rnorm(R a) { return a; }
template <>
LGF_D df rnorm<df>(df a) { return df_renorm(a); }

// Twiddles W_64^j = cos(2 pi j / 64) - i sin(2 pi j / 64), j < 64, passed by value as a kernel
// parameter (constant bank, broadcast to the warp).  Built on the host from sincospi in FP64.
template <class R>
struct Tw64 {
  R c[64];
  R s[64];
};

// W_N^k (forward: e^{-2 pi i k/N}; inverse: conjugate), N a power of two dividing 64.
template <class R, int N, bool INV>
LGF_D cx<R> twiddle(const Tw64<R> &tw, int k) {
  const int j = (k * (64 / N)) & 63;
  return INV ? cx<R>{tw.c[j], tw.s[j]} : cx<R>{tw.c[j], -tw.s[j]};
}

template <int N>
LGF_HD constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// Real product x c with the double-float error term kept unnormalised (the butterflies that follow add
// lazily); a plain product for the other arithmetics.
LGF_D double rmul_lazy(double x, double c) { return x * c; }
LGF_D float rmul_lazy(float x, float c) { return x * c; }
LGF_D df rmul_lazy(df x, df c) {
  const float p = __fmul_rn(x.hi, c.hi);
  float e = __fmaf_rn(x.hi, c.hi, -p);
  e = __fmaf_rn(x.lo, c.hi, e);
  return {p, __fmaf_rn(x.hi, c.lo, e)};
}
// v W_8^k for k = 1 or 3 (forward, W_8 = e^{-i pi/4}) or its conjugate (inverse): with s = a + b and
// d = b - a for v = a + ib and c = cos(pi/4), v W_8 = c (s + i d) and v W_8^3 = c (d - i s); the
// conjugates are c (-d + i s) and -c (s + i d).  Two sums and two real products instead of a complex
// product.
template <class R, bool INV>
LGF_D cx<R> mul_w8(cx<R> v, bool k3, const R &c) {
  const R sm = radd(v.re, v.im), d = radd(v.im, -v.re);
  const R cs = rmul_lazy(sm, c), cd = rmul_lazy(d, c);
  if (!INV) return k3 ? cx<R>{cd, -cs} : cx<R>{cs, cd};
  return k3 ? cx<R>{-cs, -cd} : cx<R>{-cd, cs};
}

// In-register radix-2 decimation-in-time FFT of length N (power of two <= 64), unnormalised.  NORM = false
// leaves double-float outputs unrenormalised (hi + lo still exact: for callers whose next operations are
// lazy sums and error-compensated products, which renormalise themselves).
template <class R, int N, bool INV, bool NORM = true>
LGF_D void fft_reg(cx<R> (&x)[N], const Tw64<R> &tw) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev<N>(i);
    if (j > i) {
      cx<R> t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= N; len <<= 1) {
#pragma unroll
    for (int i = 0; i < N; i += len) {
#pragma unroll
      for (int j = 0; j < len / 2; ++j) {
        cx<R> u = x[i + j];
        cx<R> v = x[i + j + len / 2];
        if (j * (64 / len) == 16)  // W = -i (forward) or +i (inverse): an exact swap
          v = INV ? cx<R>{-v.im, v.re} : cx<R>{v.im, -v.re};
        else if (j * (64 / len) == 8 || j * (64 / len) == 24)  // W = W_8 or W_8^3 (or conjugates)
          v = mul_w8<R, INV>(v, j * (64 / len) == 24, tw.c[8]);
        else if (j != 0)
          v = cmul(v, twiddle<R, 64, INV>(tw, j * (64 / len)));
        x[i + j] = cadd(u, v);
        x[i + j + len / 2] = csub(u, v);
      }
    }
  }
  if (NORM)
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = cnorm(x[i]);
}

// Streaming (evict-first) load of data read once, so it does not displace reused data from L2.
LGF_D double ld_stream(const double *p) { return __ldcs(p); }
LGF_D float ld_stream(const float *p) { return __ldcs(p); }
LGF_D df ld_stream(const df *p) {
  const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
  return df{v.x, v.y};
}
// complex values: one 8- or 16-byte access (cx is aligned to its size)
LGF_D cx<double> ld_stream(const cx<double> *p) {
  const double2 v = __ldcs(reinterpret_cast<const double2 *>(p));
  return cx<double>{v.x, v.y};
}
LGF_D cx<float> ld_stream(const cx<float> *p) {
  const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
  return cx<float>{v.x, v.y};
}
LGF_D cx<df> ld_stream(const cx<df> *p) {
  const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
  return cx<df>{df{v.x, v.y}, df{v.z, v.w}};
}

// ------------------------------------------------------------------ loads/stores of fields
// dtype 0: double storage, 1: float storage, 2: the kernel's own arithmetic type R (internal buffers).
template <class R>
LGF_D R load_field(const void *p, int64_t i, int dtype) {
  if (dtype == 0) return RT<R>::from(((const double *)p)[i]);
  if (dtype == 1) return RT<R>::from(((const float *)p)[i]);
  return ((const R *)p)[i];
}
template <class R>
LGF_D void store_field(void *p, int64_t i, int dtype, R v) {
  if (dtype == 0)
    ((double *)p)[i] = RT<R>::to_d(v);
  else if (dtype == 1)
    ((float *)p)[i] = RT<R>::to_f(v);
  else
    ((R *)p)[i] = v;
}
