/*
 * Plain-C FP64 oracle: H_W and per-node resolvent solves.  TEST INFRASTRUCTURE
 * ONLY -- used by tests and by the CPU-baseline leg of the benchmark, never by
 * the library.  Deliberately simple loops; no blocking, no vectorisation tricks.
 *
 * H_W = gamma5 D_W(-m0) (Eq. 1 and the definition of H_W after it), with
 *   (D_W psi)(x) = (4r + m) psi(x)
 *                - 1/2 sum_mu [ (r - g_mu) U_mu(x) psi(x+mu) + (r + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *   m = -m0, periodic space, bc_t = +1 / -1 for (anti)periodic time (sign on hops
 *   that cross the t boundary).  Chiral basis, gamma5 = diag(1,1,-1,-1):
 *   g_k = [[0, -i s_k], [i s_k, 0]] (k = x,y,z), g_t = [[0, 1], [1, 0]].
 *
 * Layouts (canonical): U[mu][t][z][y][x][3][3], psi[t][z][y][x][4][3], complex
 * interleaved (re, im).  dims = {Lx, Ly, Lz, Lt}.
 *
 * Resolvent solves (z - H_W) y = b of Eq. 6: CGNR (CG on the normal equations,
 * A = z - H_W, A^dag = conj(z) - H_W), each node on its own, OpenMP over nodes.
 * Quadrature sum: out = c0 b + sum_j c_j y_j (Eqs. 5, 7), summed in node order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const cplx I1 = I;

static void gamma_mat(int mu, cplx g[4][4]) {
  memset(g, 0, sizeof(cplx) * 16);
  switch (mu) {
    case 0: /* x */
      g[0][3] = -I1; g[1][2] = -I1; g[2][1] = I1; g[3][0] = I1; break;
    case 1: /* y */
      g[0][3] = -1; g[1][2] = 1; g[2][1] = 1; g[3][0] = -1; break;
    case 2: /* z */
      g[0][2] = -I1; g[1][3] = I1; g[2][0] = I1; g[3][1] = -I1; break;
    default: /* t */
      g[0][2] = 1; g[1][3] = 1; g[2][0] = 1; g[3][1] = 1; break;
  }
}

static long site_index(const int d[4], int x, int y, int z, int t) {
  return (((long)t * d[2] + z) * d[1] + y) * d[0] + x;
}

int oracle_hw_apply(const double* Ud, const double* ind, double* outd, const int* dims,
                    double m0, double r, int bc_t) {
  const cplx* U = (const cplx*)Ud;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
  const int* d = dims;
  long V = (long)d[0] * d[1] * d[2] * d[3];
  cplx gm[4][4][4];
  for (int mu = 0; mu < 4; ++mu) gamma_mat(mu, gm[mu]);
  for (int t = 0; t < d[3]; ++t)
    for (int z = 0; z < d[2]; ++z)
      for (int y = 0; y < d[1]; ++y)
        for (int x = 0; x < d[0]; ++x) {
          long s = site_index(d, x, y, z, t);
          cplx acc[4][3];
          for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) acc[a][c] = (4.0 * r - m0) * in[s * 12 + a * 3 + c];
          int co[4] = {x, y, z, t};
          for (int mu = 0; mu < 4; ++mu) {
            for (int dir = 0; dir < 2; ++dir) { /* 0: forward, 1: backward */
              int cn[4] = {co[0], co[1], co[2], co[3]};
              double sign = 1.0;
              if (dir == 0) {
                cn[mu] = co[mu] + 1;
                if (cn[mu] == d[mu]) { cn[mu] = 0; if (mu == 3) sign = bc_t; }
              } else {
                cn[mu] = co[mu] - 1;
                if (cn[mu] < 0) { cn[mu] = d[mu] - 1; if (mu == 3) sign = bc_t; }
              }
              long sn = site_index(d, cn[0], cn[1], cn[2], cn[3]);
              /* link: forward uses U_mu(x), backward uses U_mu(x - mu)^dag */
              const cplx* L = (dir == 0) ? &U[((long)mu * V + s) * 9] : &U[((long)mu * V + sn) * 9];
              cplx hop[4][3];
              for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                  cplx v = 0;
                  for (int j = 0; j < 3; ++j) {
                    cplx l = (dir == 0) ? L[i * 3 + j] : conj(L[j * 3 + i]);
                    v += l * in[sn * 12 + a * 3 + j];
                  }
                  hop[a][i] = sign * v;
                }
              double pm = (dir == 0) ? -1.0 : 1.0; /* (r - g) forward, (r + g) backward */
              for (int a = 0; a < 4; ++a)
                for (int c = 0; c < 3; ++c) {
                  cplx v = r * hop[a][c];
                  for (int b = 0; b < 4; ++b) v += pm * gm[mu][a][b] * hop[b][c];
                  acc[a][c] -= 0.5 * v;
                }
            }
          }
          for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) out[s * 12 + a * 3 + c] = (a < 2 ? 1.0 : -1.0) * acc[a][c];
        }
  return 0;
}

static double nrm2(const cplx* v, long n) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
  return s;
}

/* out = zs * v - H_W v */
static void shifted(const double* U, const cplx* v, cplx* out, const int* dims, double m0,
                    double r, int bc_t, cplx zs, long n) {
  oracle_hw_apply(U, (const double*)v, (double*)out, dims, m0, r, bc_t);
  for (long i = 0; i < n; ++i) out[i] = zs * v[i] - out[i];
}

int oracle_cgnr(const double* U, const double* bd, const int* dims, double m0, double r,
                int bc_t, double zre, double zim, double tol, int maxiter, double* yd,
                int* iters, double* true_relres) {
  long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  long n = 12 * V;
  const cplx* b = (const cplx*)bd;
  cplx* y = (cplx*)yd;
  cplx zz = zre + I1 * zim;
  cplx* res = malloc(sizeof(cplx) * n);
  cplx* s = malloc(sizeof(cplx) * n);
  cplx* p = malloc(sizeof(cplx) * n);
  cplx* q = malloc(sizeof(cplx) * n);
  if (!res || !s || !p || !q) { free(res); free(s); free(p); free(q); return -1; }
  for (long i = 0; i < n; ++i) { y[i] = 0; res[i] = b[i]; }
  double bn = sqrt(nrm2(b, n));
  shifted(U, res, s, dims, m0, r, bc_t, conj(zz), n);
  memcpy(p, s, sizeof(cplx) * n);
  double gam = nrm2(s, n);
  int it = 0;
  while (sqrt(nrm2(res, n)) > tol * bn && it < maxiter) {
    shifted(U, p, q, dims, m0, r, bc_t, zz, n);
    double a = gam / nrm2(q, n);
    for (long i = 0; i < n; ++i) { y[i] += a * p[i]; res[i] -= a * q[i]; }
    shifted(U, res, s, dims, m0, r, bc_t, conj(zz), n);
    double gnew = nrm2(s, n);
    double beta = gnew / gam;
    for (long i = 0; i < n; ++i) p[i] = s[i] + beta * p[i];
    gam = gnew;
    ++it;
  }
  shifted(U, y, q, dims, m0, r, bc_t, zz, n);
  for (long i = 0; i < n; ++i) q[i] = b[i] - q[i];
  *true_relres = (bn > 0) ? sqrt(nrm2(q, n)) / bn : 0.0;
  *iters = it;
  free(res); free(s); free(p); free(q);
  return it < maxiter ? 0 : 1;
}

/*
 * out = c0 b + sum_j c_j y_j with y_j from one CGNR per node.  z and c hold n
 * interleaved complex numbers.  ys (optional, may be NULL) receives every y_j,
 * node-major.  Returns 0 if every node converged.
 */
int oracle_sign_apply(const double* U, const double* bd, const int* dims, double m0, double r,
                      int bc_t, int n_nodes, const double* z, const double* c, double c0re,
                      double c0im, double tol, int maxiter, double* outd, double* ys,
                      int* iters, double* relres) {
  long n = 12L * dims[0] * dims[1] * dims[2] * dims[3];
  cplx* Y = ys ? (cplx*)ys : malloc(sizeof(cplx) * n * (long)n_nodes);
  if (!Y) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int j = 0; j < n_nodes; ++j) {
    int rc = oracle_cgnr(U, bd, dims, m0, r, bc_t, z[2 * j], z[2 * j + 1], tol, maxiter,
                         (double*)(Y + (long)j * n), &iters[j], &relres[j]);
    if (rc) bad = 1;
  }
  const cplx* b = (const cplx*)bd;
  cplx* out = (cplx*)outd;
  cplx c0 = c0re + I1 * c0im;
  for (long i = 0; i < n; ++i) out[i] = c0 * b[i];
  for (int j = 0; j < n_nodes; ++j) {
    cplx cj = c[2 * j] + I1 * c[2 * j + 1];
    const cplx* yj = Y + (long)j * n;
    for (long i = 0; i < n; ++i) out[i] += cj * yj[i];
  }
  if (!ys) free(Y);
  return bad;
}

/*
 * The same quadrature sum for several sources at once: out_r = c0 b_r + sum_j c_j y_{r,j}
 * with one CGNR per (source, node) pair, OpenMP over all pairs (so that a few nodes of
 * many sources fill the cores).  b and out hold nsrc canonical spinors back to back;
 * iters and relres receive nsrc * n_nodes entries, source-major.  Returns 0 if every
 * solve converged.
 */
int oracle_sign_apply_many(const double* U, const double* bd, const int* dims, double m0, double r,
                           int bc_t, int nsrc, int n_nodes, const double* z, const double* c,
                           double c0re, double c0im, double tol, int maxiter, double* outd,
                           int* iters, double* relres) {
  long n = 12L * dims[0] * dims[1] * dims[2] * dims[3];
  long npair = (long)nsrc * n_nodes;
  cplx* Y = malloc(sizeof(cplx) * n * (npair > 0 ? npair : 1));
  if (!Y) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (long q = 0; q < npair; ++q) {
    long rr = q / n_nodes, j = q % n_nodes;
    int rc = oracle_cgnr(U, bd + 2 * rr * n, dims, m0, r, bc_t, z[2 * j], z[2 * j + 1], tol, maxiter,
                         (double*)(Y + q * n), &iters[q], &relres[q]);
    if (rc) bad = 1;
  }
  cplx c0 = c0re + I1 * c0im;
  for (long rr = 0; rr < nsrc; ++rr) {
    const cplx* b = (const cplx*)bd + rr * n;
    cplx* out = (cplx*)outd + rr * n;
    for (long i = 0; i < n; ++i) out[i] = c0 * b[i];
    for (int j = 0; j < n_nodes; ++j) {
      cplx cj = c[2 * j] + I1 * c[2 * j + 1];
      const cplx* yj = Y + (rr * n_nodes + j) * n;
      for (long i = 0; i < n; ++i) out[i] += cj * yj[i];
    }
  }
  free(Y);
  return bad;
}
