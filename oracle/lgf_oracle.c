/*
 * lgf_oracle.c -- plain, slow FP64 CPU oracle for the LGF Poisson / heat-kernel path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (paper: Yu, Dorschner & Colonius, "Multi-resolution lattice Green's
 * function method for incompressible flows", Sec. 2.2-2.3):
 *
 *   * the 7-point lattice Green's function G with L G = delta (Sec. 2.2, Eq. (eq:discrete_laplace)
 *     and (eq:lgf_convolution)), evaluated from the Bessel-product integral
 *         G(n) = - int_0^inf  prod_i  e^{-2t} I_{n_i}(2t)  dt
 *     by composite Gauss-Legendre quadrature in t on [0,1] and in u = ln t on [1,T], plus the
 *     term-by-term integrated large-argument (Hankel) series of e^{-x} I_nu(x) on [T, inf);
 *   * scaled modified Bessel functions e^{-x} I_k(x), k = 0..kmax, by Miller's backward
 *     recurrence normalised with  e^{-x} (I_0 + 2 sum_k I_k) = 1;
 *   * the direct O(N_t N_s) lattice convolution  out(n) = scale * sum_m K(n-m) f(m)  with
 *     Neumaier-compensated sums (Eq. (eq:lgf_convolution) for K = G; the heat kernel
 *     E_alpha(n) = prod_i e^{-2 alpha} I_{|n_i|}(2 alpha) of Sec. 2.3, Eq. (eq:IF-single), for K = E).
 *
 * Built with -O2 -fopenmp -ffp-contract=off (no fast-math): every rounding is a plain FP64 one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ---- Gauss-Legendre rule on [-1,1]: Newton iteration on P_n(x) via its three-term recurrence. */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ---- e^{-x} I_k(x) for k = 0..kmax (Miller backward recurrence, sum normalisation). */
void oracle_ive_all(double x, int kmax, double *out) {
  for (int k = 0; k <= kmax; ++k) out[k] = 0.0;
  if (x <= 0.0) {
    out[0] = 1.0;
    return;
  }
  double start = sqrt((double)kmax * kmax + 80.0 * x) + 40.0;
  int M = (int)start;
  if (M <= kmax) M = kmax + 40;
  double bp = 0.0, b = 1.0; /* b_{k+1}, b_k with k = M */
  double sum = 0.0;         /* sum_{j >= 1} b_j, accumulated downward */
  for (int k = M; k >= 1; --k) {
    if (k <= kmax) out[k] = b;
    sum += b;
    double bm = (2.0 * k / x) * b + bp;
    bp = b;
    b = bm;
    if (fabs(b) > 1e200) {
      const double s = 1e-200;
      b *= s;
      bp *= s;
      sum *= s;
      int hi = kmax < M ? kmax : M;
      for (int j = k; j <= hi; ++j) out[j] *= s;
    }
  }
  out[0] = b;
  double norm = b + 2.0 * sum;
  for (int k = 0; k <= kmax; ++k) out[k] /= norm;
}

/* Neumaier accumulate */
static inline void neu_add(double *s, double *c, double v) {
  double t = *s + v;
  if (fabs(*s) >= fabs(v))
    *c += (*s - t) + v;
  else
    *c += (v - t) + *s;
  *s = t;
}

/* Coefficients of the large-argument series of e^{-x} I_nu(x) written in t with x = 2t:
 *   e^{-2t} I_nu(2t) ~ (4 pi t)^{-1/2} sum_k alpha_k t^{-k},
 *   alpha_k = (-1)^k a_k(nu) / 2^k,  a_k = prod_{j<=k} (4 nu^2 - (2j-1)^2) / (k! 8^k). */
#define ORACLE_TAIL_TERMS 10
static void hankel_alpha(int nu, double *alpha) {
  double a = 1.0;
  alpha[0] = 1.0;
  for (int k = 1; k < ORACLE_TAIL_TERMS; ++k) {
    a *= (4.0 * nu * nu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
    alpha[k] = ((k & 1) ? -a : a) / ldexp(1.0, k);
  }
}

/* int_T^inf prod_i e^{-2t} I_{n_i}(2t) dt from the product of the three series. */
static double tail_integral(int n1, int n2, int n3, double T) {
  double a1[ORACLE_TAIL_TERMS], a2[ORACLE_TAIL_TERMS], a3[ORACLE_TAIL_TERMS];
  hankel_alpha(n1, a1);
  hankel_alpha(n2, a2);
  hankel_alpha(n3, a3);
  double total = 0.0;
  for (int j = 0; j < ORACLE_TAIL_TERMS; ++j) {
    double cj = 0.0;
    for (int p = 0; p <= j; ++p)
      for (int q = 0; q <= j - p; ++q) cj += a1[p] * a2[q] * a3[j - p - q];
    total += cj * pow(T, -0.5 - j) / (j + 0.5);
  }
  return total * pow(4.0 * ORACLE_PI, -1.5);
}

/* Quadrature rule for the table: nodes t_j and weights w_j of int_0^T f(t) dt. */
static int build_rule(int nmax, double T, double **t_out, double **w_out) {
  const int ng = 20;
  double gx[20], gw[20];
  gauss_legendre(ng, gx, gw);
  double lnT = log(T);
  const double du = 0.25;
  int npan_u = (int)ceil(lnT / du);
  int nnodes = 2 * ng + npan_u * ng;
  double *t = (double *)malloc(sizeof(double) * nnodes);
  double *w = (double *)malloc(sizeof(double) * nnodes);
  int m = 0;
  /* [0,1] in t: two panels */
  for (int p = 0; p < 2; ++p) {
    double a = 0.5 * p, b = a + 0.5;
    for (int i = 0; i < ng; ++i) {
      t[m] = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
      w[m] = 0.5 * (b - a) * gw[i];
      ++m;
    }
  }
  /* [1,T] in u = ln t: dt = t du */
  double hu = lnT / npan_u;
  for (int p = 0; p < npan_u; ++p) {
    double a = p * hu, b = a + hu;
    for (int i = 0; i < ng; ++i) {
      double u = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
      t[m] = exp(u);
      w[m] = 0.5 * (b - a) * gw[i] * t[m];
      ++m;
    }
  }
  (void)nmax;
  *t_out = t;
  *w_out = w;
  return nnodes;
}

/*
 * Dense first-octant table: G[(c*(nmax+1) + b)*(nmax+1) + a] = G(a,b,c) for 0 <= a,b,c <= nmax.
 * Only the sorted triples a <= b <= c are integrated; the rest are filled by the octahedral
 * symmetry of the 7-point Laplacian.  Returns the number of quadrature nodes used.
 */
int oracle_lgf_table(int nmax, double *G) {
  if (nmax < 0) return -1;
  double T = 2000.0 * (nmax > 1 ? (double)nmax * nmax : 1.0);
  if (T < 2000.0) T = 2000.0;
  double *t, *w;
  int nn = build_rule(nmax, T, &t, &w);
  const int K = nmax + 1;
  double *iv = (double *)malloc(sizeof(double) * (size_t)nn * K);
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < nn; ++j) oracle_ive_all(2.0 * t[j], nmax, iv + (size_t)j * K);

#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c <= nmax; ++c) {
    for (int b = 0; b <= c; ++b) {
      for (int a = 0; a <= b; ++a) {
        double s = 0.0, comp = 0.0;
        for (int j = 0; j < nn; ++j) {
          const double *r = iv + (size_t)j * K;
          neu_add(&s, &comp, w[j] * (r[a] * r[b] * r[c]));
        }
        neu_add(&s, &comp, tail_integral(a, b, c, T));
        double g = -(s + comp);
        int p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
        for (int q = 0; q < 6; ++q)
          G[((size_t)p[q][2] * K + p[q][1]) * K + p[q][0]] = g;
      }
    }
  }
  free(iv);
  free(t);
  free(w);
  return nn;
}

/* Single value of G (same rule as the table), for spot checks far from the origin. */
double oracle_lgf_value(int n1, int n2, int n3) {
  n1 = abs(n1);
  n2 = abs(n2);
  n3 = abs(n3);
  int nmax = n1 > n2 ? n1 : n2;
  nmax = nmax > n3 ? nmax : n3;
  double T = 2000.0 * (nmax > 1 ? (double)nmax * nmax : 1.0);
  if (T < 2000.0) T = 2000.0;
  double *t, *w;
  int nn = build_rule(nmax, T, &t, &w);
  double *r = (double *)malloc(sizeof(double) * (nmax + 1));
  double s = 0.0, comp = 0.0;
  for (int j = 0; j < nn; ++j) {
    oracle_ive_all(2.0 * t[j], nmax, r);
    neu_add(&s, &comp, w[j] * (r[n1] * r[n2] * r[n3]));
  }
  neu_add(&s, &comp, tail_integral(n1, n2, n3, T));
  free(r);
  free(t);
  free(w);
  return -(s + comp);
}

/*
 * Direct lattice convolution with the dense first-octant kernel K (extent kn per axis,
 * K[(|dz|*kn + |dy|)*kn + |dx|]); kernel entries beyond the extent count as zero (used for the
 * compactly supported heat kernel; the LGF table must cover every offset, which the caller checks).
 *   out[c*ntgt + i] = scale * sum_j K(tgt_i - src_j) * val[c*nsrc + j]
 * Neumaier-compensated, OpenMP over targets.
 */
void oracle_direct_conv(const double *Kt, int kn, int nsrc, const int32_t *src_xyz,
                        const double *val, int ntgt, const int32_t *tgt_xyz, int ncomp,
                        double scale, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < ntgt; ++i) {
    const int tx = tgt_xyz[3 * i], ty = tgt_xyz[3 * i + 1], tz = tgt_xyz[3 * i + 2];
    for (int c = 0; c < ncomp; ++c) {
      double s = 0.0, comp = 0.0;
      const double *v = val + (size_t)c * nsrc;
      for (int j = 0; j < nsrc; ++j) {
        int dx = abs(tx - src_xyz[3 * j]);
        int dy = abs(ty - src_xyz[3 * j + 1]);
        int dz = abs(tz - src_xyz[3 * j + 2]);
        if (dx >= kn || dy >= kn || dz >= kn) continue;
        double kv = Kt[((size_t)dz * kn + dy) * kn + dx];
        neu_add(&s, &comp, kv * v[j]);
      }
      out[(size_t)c * ntgt + i] = scale * (s + comp);
    }
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Compactly supported stencil convolution on a dense box (used for the heat kernel, Sec. 2.3):
 *   out(n) = sum_{|d_i| <= r} K(d) src(n - d),   src = 0 outside the box,
 * K given in full on [-r, r]^3 as K[((dz+r)*(2r+1) + dy+r)*(2r+1) + dx+r].  Arrays are [nz][ny][nx].
 */
void oracle_box_stencil_conv(const double *Kf, int r, const double *src, int nz, int ny, int nx,
                             double *out) {
  const int w = 2 * r + 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z) {
    for (int y = 0; y < ny; ++y) {
      for (int x = 0; x < nx; ++x) {
        double s = 0.0, comp = 0.0;
        for (int dz = -r; dz <= r; ++dz) {
          int sz = z - dz;
          if (sz < 0 || sz >= nz) continue;
          for (int dy = -r; dy <= r; ++dy) {
            int sy = y - dy;
            if (sy < 0 || sy >= ny) continue;
            for (int dx = -r; dx <= r; ++dx) {
              int sx = x - dx;
              if (sx < 0 || sx >= nx) continue;
              double v = src[((size_t)sz * ny + sy) * nx + sx];
              if (v == 0.0) continue;
              neu_add(&s, &comp, Kf[((size_t)(dz + r) * w + (dy + r)) * w + (dx + r)] * v);
            }
          }
        }
        out[((size_t)z * ny + y) * nx + x] = s + comp;
      }
    }
  }
}
