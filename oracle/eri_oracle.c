/*
 * CPU oracle for contracted Gaussian electron repulsion integrals (ab|cd).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference the CUDA path is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never calls it and shares no code, header, table or constant with it.
 *
 * What it computes (FusionRCG paper, Sec. II-A): the contracted ERI of Eq. 1
 * over Cartesian Gaussians, by the Head-Gordon-Pople two-phase scheme:
 *   Phase 1, Eq. 2: Obara-Saika vertical recurrence (VRR) on [e0|f0]^(m),
 *            started from the Boys-function base values;
 *   contraction: accumulate-then-transform (Sec. III-C-1, Algorithm 2);
 *   Phase 2, Eq. 3: horizontal recurrence (HRR) on the bra, then the ket;
 *   Cartesian-to-spherical transform of Eq. 8, applied AFTER both HRR sweeps
 *   (materialize-then-transform, Eq. 17) -- deliberately not the stepwise
 *   fusion of Eq. 16 that the CUDA path uses.
 * The recurrence axis is always the first non-zero Cartesian component in
 * x -> y -> z order, bra VRR first, then ket VRR (the conventional order of
 * the paper's ablation, Sec. V-B) -- deliberately different from the CUDA
 * path's axis rule.
 *
 * Readings of the paper taken here (the paper is silent or garbled on them):
 *  - Eq. 2's third term is the standard Obara-Saika one,
 *      (a_i / 2 zeta) ( [a-1_i 0|c 0]^(m) - (rho/zeta) [a-1_i 0|c 0]^(m+1) );
 *    the ket recurrence is its mirror image with eta, Q, C.
 *  - The base values are [00|00]^(m) = 2 pi^(5/2) / (zeta eta sqrt(zeta+eta))
 *      K_AB K_CD F_m(T), K_AB = exp(-a_a a_b |A-B|^2 / zeta).
 *  - zeta, eta, rho, P, Q, W, T take their textbook meaning.
 *  - Primitive normalisation N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!)
 *    (the norm of x^l exp(-a r^2)), shared by every Cartesian component of a
 *    shell; contracted functions are not renormalised.
 *  - Cartesian order: x exponent descending, then y descending.
 *  - Spherical functions: real solid harmonics, Racah normalised, no
 *    Condon-Shortley phase, m = -l..l.
 *  - Boys function: power series plus downward recursion for T <= 50;
 *    erf plus upward recursion above.
 *
 * Compiled twice: with REAL = double (the timed oracle) and with
 * REAL = long double (symbol prefix oracle_ld_) to adjudicate disagreements
 * caused by rounding.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifdef ORACLE_LONG_DOUBLE
typedef long double real;
#define R(x) x##L
#define R_EXP expl
#define R_SQRT sqrtl
#define R_ERF erfl
#define R_FABS fabsl
#define R_POW powl
#define OFN(name) oracle_ld_##name
#else
typedef double real;
#define R(x) x
#define R_EXP exp
#define R_SQRT sqrt
#define R_ERF erf
#define R_FABS fabs
#define R_POW pow
#define OFN(name) oracle_##name
#endif

#define LMAX 4                      /* highest shell angular momentum */
#define LSUM_MAX (4 * LMAX)         /* highest Boys order needed */
#define NCART(l) (((l) + 1) * ((l) + 2) / 2)
#define NCUM(n) (((n) + 1) * ((n) + 2) * ((n) + 3) / 6) /* Cartesian tuples with |e| <= n */
#define NE_MAX NCUM(2 * LMAX)
static const real PI = R(3.14159265358979323846264338327950288);

/* ------------------------------------------------------------------------- */
/* Cartesian component bookkeeping                                            */
/* ------------------------------------------------------------------------- */

/* Index of (i,j,k), i+j+k = l, within its shell: x exponent descending, then
 * y descending (xx, xy, xz, yy, yz, zz). */
static int cart_index(int i, int j, int k) {
  (void)i;
  int jk = j + k;
  return jk * (jk + 1) / 2 + k;
}

/* Index among all tuples with |e| <= n, shells stacked by total degree. */
static int cum_index(const int e[3]) {
  int n = e[0] + e[1] + e[2];
  return (n == 0 ? 0 : NCUM(n - 1)) + cart_index(e[0], e[1], e[2]);
}

/* The c-th Cartesian tuple of degree l, in the order above. */
static void cart_tuple(int l, int c, int e[3]) {
  int n = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      if (n == c) {
        e[0] = i;
        e[1] = j;
        e[2] = l - i - j;
        return;
      }
      ++n;
    }
}

static int first_nonzero(const int e[3]) {
  for (int i = 0; i < 3; ++i)
    if (e[i] > 0) return i;
  return -1;
}

static real dfact(int n) { /* n!! with (-1)!! = 0!! = 1 */
  real r = 1;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

static real fact(int n) {
  real r = 1;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}

static real binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  return fact(n) / (fact(k) * fact(n - k));
}

/* ------------------------------------------------------------------------- */
/* Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt, m = 0..L             */
/* (base values of Phase 1, Sec. II-A; Algorithm 2 step "Boys")              */
/* ------------------------------------------------------------------------- */
void OFN(boys)(int L, real T, real* F) {
  if (T <= R(50.0)) {
    /* F_L(T) = exp(-T) sum_k (2T)^k / ((2L+1)(2L+3)...(2L+2k+1)) */
    real term = R(1.0) / (2 * L + 1), sum = term;
    for (int k = 1; k < 2000; ++k) {
      term *= (2 * T) / (2 * L + 2 * k + 1);
      sum += term;
      if (term < sum * R(1e-40)) break;
    }
    real ex = R_EXP(-T);
    F[L] = ex * sum;
    /* downward: F_m = (2T F_{m+1} + exp(-T)) / (2m+1) */
    for (int m = L - 1; m >= 0; --m) F[m] = (2 * T * F[m + 1] + ex) / (2 * m + 1);
  } else {
    /* F_0 = (1/2) sqrt(pi/T) erf(sqrt T); upward F_{m+1} = ((2m+1)F_m - e^-T)/(2T) */
    real ex = R_EXP(-T);
    F[0] = R(0.5) * R_SQRT(PI / T) * R_ERF(R_SQRT(T));
    for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - ex) / (2 * T);
  }
}

/* ------------------------------------------------------------------------- */
/* Cartesian -> spherical coefficients t^(l)_{m,ijk} of Eq. 8                 */
/* Real solid harmonics from their closed-form expansion (Helgaker, Jorgensen */
/* and Olsen, Molecular Electronic-Structure Theory, Eqs. 6.4.47-6.4.50),     */
/* Racah normalised, so that with every Cartesian component normalised like   */
/* x^l the spherical functions are normalised.  Row m+l, column cart_index.   */
/* ------------------------------------------------------------------------- */
void OFN(cart2sph)(int l, real* T) {
  int nc = NCART(l);
  memset(T, 0, sizeof(real) * (2 * l + 1) * nc);
  for (int m = -l; m <= l; ++m) {
    int am = m < 0 ? -m : m;
    /* v runs over integers (m >= 0) or half-integers (m < 0); use w = 2v */
    int wm = m < 0 ? 1 : 0;
    real Nlm = R_SQRT(2 * fact(l + am) * fact(l - am) / (m == 0 ? R(2.0) : R(1.0))) /
               (fact(l) * (real)(1 << am));
    for (int t = 0; t <= (l - am) / 2; ++t)
      for (int u = 0; u <= t; ++u)
        for (int w = wm; w <= am; w += 2) { /* 2v from v_m to floor(|m|/2 - v_m) + v_m */
          int sgn_exp = t + (w - wm) / 2;
          real c = ((sgn_exp & 1) ? -1 : 1) * binom(l, t) * binom(l - t, am + t) * binom(t, u) * binom(am, w);
          for (int q = 0; q < t; ++q) c *= R(0.25);
          int px = 2 * t + am - 2 * u - w;
          int py = 2 * u + w;
          int pz = l - 2 * t - am;
          if (px < 0 || py < 0 || pz < 0) continue;
          T[(m + l) * nc + cart_index(px, py, pz)] += Nlm * c;
        }
  }
}

/* N(a, l): norm of x^l exp(-a r^2). */
static real prim_norm(real a, int l) {
  return R_POW(2 * a / PI, R(0.75)) * R_POW(4 * a, R(0.5) * l) / R_SQRT(dfact(2 * l - 1));
}

/* ------------------------------------------------------------------------- */
/* One contracted shell quartet                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
  int l;
  int nprim;
  const double* exps;
  const double* coefs;
  real ctr[3];
} oshell;

/* Phase 1 working table [m][e][f], e and f over all tuples with |e| <= la+lb,
 * |f| <= lc+ld. */
typedef struct {
  int ne, nf, nm;
  real* v;
  real* H; /* contracted [e0|f0] targets, [e][f] */
} vrr_table;

#define VIDX(t, m, ie, jf) ((((size_t)(m) * (t)->ne) + (ie)) * (t)->nf + (jf))

/* Eq. 2 and its ket mirror for one primitive quartet, added into t->H. */
static void primitive_vrr(vrr_table* t, int lab, int lcd, int lmin_e, int lmin_f, real za, real zb, real zc,
                          real zd, const real A[3], const real B[3], const real C[3], const real D[3],
                          real scale) {
  int L = lab + lcd;
  real zeta = za + zb, eta = zc + zd;
  real P[3], Q[3], W[3], PA[3], WP[3], QC[3], WQ[3];
  real ab2 = 0, cd2 = 0, pq2 = 0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (za * A[i] + zb * B[i]) / zeta;
    Q[i] = (zc * C[i] + zd * D[i]) / eta;
    W[i] = (zeta * P[i] + eta * Q[i]) / (zeta + eta);
    PA[i] = P[i] - A[i];
    WP[i] = W[i] - P[i];
    QC[i] = Q[i] - C[i];
    WQ[i] = W[i] - Q[i];
    ab2 += (A[i] - B[i]) * (A[i] - B[i]);
    cd2 += (C[i] - D[i]) * (C[i] - D[i]);
    pq2 += (P[i] - Q[i]) * (P[i] - Q[i]);
  }
  real rho = zeta * eta / (zeta + eta);
  real T = rho * pq2;
  real Kab = R_EXP(-za * zb / zeta * ab2);
  real Kcd = R_EXP(-zc * zd / eta * cd2);
  real pref = 2 * R_SQRT(PI) * PI * PI / (zeta * eta * R_SQRT(zeta + eta)) * Kab * Kcd * scale;
  real F[LSUM_MAX + 1];
  OFN(boys)(L, T, F);

  /* [00|00]^(m) */
  for (int m = 0; m <= L; ++m) t->v[VIDX(t, m, 0, 0)] = pref * F[m];

  /* bra VRR: [e0|00]^(m), |e| = 1..lab, m <= L - |e| */
  for (int n = 1; n <= lab; ++n)
    for (int c = 0; c < NCART(n); ++c) {
      int e[3];
      cart_tuple(n, c, e);
      int i = first_nonzero(e);
      int e1[3] = {e[0], e[1], e[2]}, e2[3];
      e1[i] -= 1;
      memcpy(e2, e1, sizeof e2);
      e2[i] -= 1;
      int ie = cum_index(e), ie1 = cum_index(e1), ie2 = e2[i] >= 0 ? cum_index(e2) : -1;
      for (int m = 0; m <= L - n; ++m) {
        real val = PA[i] * t->v[VIDX(t, m, ie1, 0)] + WP[i] * t->v[VIDX(t, m + 1, ie1, 0)];
        if (ie2 >= 0)
          val += (e1[i]) / (2 * zeta) * (t->v[VIDX(t, m, ie2, 0)] - rho / zeta * t->v[VIDX(t, m + 1, ie2, 0)]);
        t->v[VIDX(t, m, ie, 0)] = val;
      }
    }

  /* ket VRR: [e0|f0]^(m), |f| = 1..lcd, every |e| <= lab, m <= L - |e| - |f| */
  for (int nf = 1; nf <= lcd; ++nf)
    for (int cf = 0; cf < NCART(nf); ++cf) {
      int f[3];
      cart_tuple(nf, cf, f);
      int i = first_nonzero(f);
      int f1[3] = {f[0], f[1], f[2]}, f2[3];
      f1[i] -= 1;
      memcpy(f2, f1, sizeof f2);
      f2[i] -= 1;
      int jf = cum_index(f), jf1 = cum_index(f1), jf2 = f2[i] >= 0 ? cum_index(f2) : -1;
      for (int ne = 0; ne <= lab; ++ne)
        for (int ce = 0; ce < NCART(ne); ++ce) {
          int e[3];
          cart_tuple(ne, ce, e);
          int ie = cum_index(e);
          int em[3] = {e[0], e[1], e[2]};
          em[i] -= 1;
          int iem = em[i] >= 0 ? cum_index(em) : -1;
          for (int m = 0; m <= L - ne - nf; ++m) {
            real val = QC[i] * t->v[VIDX(t, m, ie, jf1)] + WQ[i] * t->v[VIDX(t, m + 1, ie, jf1)];
            if (jf2 >= 0)
              val += (f1[i]) / (2 * eta) * (t->v[VIDX(t, m, ie, jf2)] - rho / eta * t->v[VIDX(t, m + 1, ie, jf2)]);
            if (iem >= 0) val += e[i] / (2 * (zeta + eta)) * t->v[VIDX(t, m + 1, iem, jf1)];
            t->v[VIDX(t, m, ie, jf)] = val;
          }
        }
    }

  /* contraction (accumulate-then-transform): H[e][f] += [e0|f0]^(0) */
  for (int ne = lmin_e; ne <= lab; ++ne)
    for (int ce = 0; ce < NCART(ne); ++ce) {
      int e[3];
      cart_tuple(ne, ce, e);
      int ie = cum_index(e);
      for (int nf = lmin_f; nf <= lcd; ++nf)
        for (int cf = 0; cf < NCART(nf); ++cf) {
          int f[3];
          cart_tuple(nf, cf, f);
          int jf = cum_index(f);
          t->H[(size_t)ie * t->nf + jf] += t->v[VIDX(t, 0, ie, jf)];
        }
    }
}

/* Eq. 3 on one centre pair: from X0[e] (|e| in [l1, l1+l2]) build (a b) for
 * |a| = l1, |b| = l2, written to out[ca * NCART(l2) + cb].  X0 is indexed by
 * cum_index over |e| <= l1 + l2; stride lets the caller pass a strided view. */
static void hrr_pair(int l1, int l2, const real AB[3], const real* X0, size_t stride, real* out) {
  int n12 = l1 + l2;
  /* level j holds (e, b) with |b| = j and |e| in [l1, n12 - j] */
  real* lev[LMAX + 1];
  int ncum = NCUM(n12);
  for (int j = 0; j <= l2; ++j) lev[j] = (real*)calloc((size_t)ncum * NCART(j), sizeof(real));
  for (int ie = 0; ie < ncum; ++ie) lev[0][ie] = X0[(size_t)ie * stride];
  for (int j = 1; j <= l2; ++j)
    for (int ne = l1; ne <= n12 - j; ++ne)
      for (int ce = 0; ce < NCART(ne); ++ce) {
        int e[3];
        cart_tuple(ne, ce, e);
        int ie = cum_index(e);
        for (int cb = 0; cb < NCART(j); ++cb) {
          int b[3];
          cart_tuple(j, cb, b);
          int i = first_nonzero(b);
          int bm[3] = {b[0], b[1], b[2]};
          bm[i] -= 1;
          int ep[3] = {e[0], e[1], e[2]};
          ep[i] += 1;
          int cbm = cart_index(bm[0], bm[1], bm[2]);
          /* (e, b) = (e + 1_i, b - 1_i) + AB_i (e, b - 1_i) */
          lev[j][(size_t)ie * NCART(j) + cb] = lev[j - 1][(size_t)cum_index(ep) * NCART(j - 1) + cbm] +
                                               AB[i] * lev[j - 1][(size_t)ie * NCART(j - 1) + cbm];
        }
      }
  int off = l1 == 0 ? 0 : NCUM(l1 - 1);
  for (int ca = 0; ca < NCART(l1); ++ca)
    for (int cb = 0; cb < NCART(l2); ++cb) out[ca * NCART(l2) + cb] = lev[l2][(size_t)(off + ca) * NCART(l2) + cb];
  for (int j = 0; j <= l2; ++j) free(lev[j]);
}

/* Apply the one-index transform M (rows nr, cols n_in) to index `which` of a
 * 4-index row-major tensor of dims d[4]; result dims with d[which] = nr. */
static void transform_index(const real* in, const int d[4], int which, const real* M, int nr, real* out) {
  int dout[4] = {d[0], d[1], d[2], d[3]};
  dout[which] = nr;
  for (int i0 = 0; i0 < dout[0]; ++i0)
    for (int i1 = 0; i1 < dout[1]; ++i1)
      for (int i2 = 0; i2 < dout[2]; ++i2)
        for (int i3 = 0; i3 < dout[3]; ++i3) {
          int io[4] = {i0, i1, i2, i3};
          real s = 0;
          for (int k = 0; k < d[which]; ++k) {
            int ii[4] = {i0, i1, i2, i3};
            ii[which] = k;
            s += M[io[which] * d[which] + k] * in[((ii[0] * d[1] + ii[1]) * d[2] + ii[2]) * d[3] + ii[3]];
          }
          out[((i0 * dout[1] + i1) * dout[2] + i2) * dout[3] + i3] = s;
        }
}

/* The contracted block (ab|cd) for one shell quartet in the caller's index
 * order, row-major; spherical (cart == 0) or Cartesian (cart == 1). */
static void shell_quartet(const oshell* sa, const oshell* sb, const oshell* sc, const oshell* sd, int cart,
                          double* out) {
  int la = sa->l, lb = sb->l, lc = sc->l, ld = sd->l;
  int lab = la + lb, lcd = lc + ld;
  vrr_table t;
  t.ne = NCUM(lab);
  t.nf = NCUM(lcd);
  t.nm = lab + lcd + 1;
  t.v = (real*)calloc((size_t)t.nm * t.ne * t.nf, sizeof(real));
  t.H = (real*)calloc((size_t)t.ne * t.nf, sizeof(real));

  for (int pa = 0; pa < sa->nprim; ++pa)
    for (int pb = 0; pb < sb->nprim; ++pb)
      for (int pc = 0; pc < sc->nprim; ++pc)
        for (int pd = 0; pd < sd->nprim; ++pd) {
          real za = sa->exps[pa], zb = sb->exps[pb], zc = sc->exps[pc], zd = sd->exps[pd];
          real scale = (real)sa->coefs[pa] * prim_norm(za, la) * (real)sb->coefs[pb] * prim_norm(zb, lb) *
                       (real)sc->coefs[pc] * prim_norm(zc, lc) * (real)sd->coefs[pd] * prim_norm(zd, ld);
          primitive_vrr(&t, lab, lcd, la, lc, za, zb, zc, zd, sa->ctr, sb->ctr, sc->ctr, sd->ctr, scale);
        }

  real AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = sa->ctr[i] - sb->ctr[i];
    CD[i] = sc->ctr[i] - sd->ctr[i];
  }
  int na = NCART(la), nb = NCART(lb), nc = NCART(lc), nd = NCART(ld);
  /* bra HRR for every ket tuple f: G1[f][a][b] */
  real* G1 = (real*)calloc((size_t)t.nf * na * nb, sizeof(real));
  for (int jf = 0; jf < t.nf; ++jf) hrr_pair(la, lb, AB, t.H + jf, (size_t)t.nf, G1 + (size_t)jf * na * nb);
  /* ket HRR for every bra pair (a,b): cartesian (ab|cd) */
  real* cartb = (real*)calloc((size_t)na * nb * nc * nd, sizeof(real));
  real* tmp = (real*)malloc(sizeof(real) * nc * nd);
  for (int ab = 0; ab < na * nb; ++ab) {
    hrr_pair(lc, ld, CD, G1 + ab, (size_t)na * nb, tmp);
    for (int k = 0; k < nc * nd; ++k) cartb[(size_t)ab * nc * nd + k] = tmp[k];
  }
  free(tmp);

  if (cart) {
    for (int k = 0; k < na * nb * nc * nd; ++k) out[k] = (double)cartb[k];
  } else {
    /* materialize-then-transform, Eq. 17: (T_a x T_b x T_c x T_d) applied
     * to the full Cartesian tensor, one index after another */
    int ls[4] = {la, lb, lc, ld};
    int d[4] = {na, nb, nc, nd};
    real* cur = cartb;
    for (int w = 0; w < 4; ++w) {
      int nr = 2 * ls[w] + 1;
      real* M = (real*)malloc(sizeof(real) * nr * d[w]);
      OFN(cart2sph)(ls[w], M);
      int dn[4] = {d[0], d[1], d[2], d[3]};
      dn[w] = nr;
      real* nxt = (real*)calloc((size_t)dn[0] * dn[1] * dn[2] * dn[3], sizeof(real));
      transform_index(cur, d, w, M, nr, nxt);
      free(M);
      free(cur);
      cur = nxt;
      memcpy(d, dn, sizeof d);
    }
    for (int k = 0; k < d[0] * d[1] * d[2] * d[3]; ++k) out[k] = (double)cur[k];
    cartb = cur;
  }
  free(cartb);
  free(G1);
  free(t.v);
  free(t.H);
}

/* ------------------------------------------------------------------------- */
/* Batch driver                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
  const int *shell_l, *shell_nprim, *shell_center, *shell_prim;
  const double *centers, *exps, *coefs;
  const int* quartets;
  const long long* offsets;
  double* out;
  int cart;
  long long next; /* shared work counter */
  long long nq;
  pthread_mutex_t mu;
} batch_job;

static void make_shell(const batch_job* j, int s, oshell* o) {
  o->l = j->shell_l[s];
  o->nprim = j->shell_nprim[s];
  o->exps = j->exps + j->shell_prim[s];
  o->coefs = j->coefs + j->shell_prim[s];
  for (int i = 0; i < 3; ++i) o->ctr[i] = j->centers[3 * j->shell_center[s] + i];
}

static void* batch_worker(void* arg) {
  batch_job* j = (batch_job*)arg;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    long long q = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (q >= j->nq) break;
    oshell s[4];
    for (int k = 0; k < 4; ++k) make_shell(j, j->quartets[4 * q + k], &s[k]);
    shell_quartet(&s[0], &s[1], &s[2], &s[3], j->cart, j->out + j->offsets[q]);
  }
  return NULL;
}

/* Contracted ERIs for nq quartets (shell indices quartets[4q..4q+3], taken
 * in the given order), block q written at out + offsets[q].  Returns 0, or -1
 * on an argument error (l out of range, bad index, non-positive exponent). */
int OFN(eri_batch)(const int* shell_l, const int* shell_nprim, const int* shell_center, const int* shell_prim,
                   int nshell, const double* centers, const double* exps, const double* coefs,
                   const int* quartets, long long nq, int cart, const long long* offsets, double* out,
                   int nthreads) {
  for (long long q = 0; q < nq; ++q)
    for (int k = 0; k < 4; ++k) {
      int s = quartets[4 * q + k];
      if (s < 0 || s >= nshell || shell_l[s] < 0 || shell_l[s] > LMAX || shell_nprim[s] < 1) return -1;
      for (int p = 0; p < shell_nprim[s]; ++p)
        if (!(exps[shell_prim[s] + p] > 0)) return -1;
    }
  batch_job j;
  j.shell_l = shell_l;
  j.shell_nprim = shell_nprim;
  j.shell_center = shell_center;
  j.shell_prim = shell_prim;
  j.centers = centers;
  j.exps = exps;
  j.coefs = coefs;
  j.quartets = quartets;
  j.offsets = offsets;
  j.out = out;
  j.cart = cart;
  j.next = 0;
  j.nq = nq;
  pthread_mutex_init(&j.mu, NULL);
  if (nthreads <= 1) {
    batch_worker(&j);
  } else {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &j);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
  }
  pthread_mutex_destroy(&j.mu);
  return 0;
}

/* Boys values as double, for the tests. */
void OFN(boys_d)(int L, double T, double* F) {
  real Fr[LSUM_MAX + 64];
  OFN(boys)(L, (real)T, Fr);
  for (int m = 0; m <= L; ++m) F[m] = (double)Fr[m];
}

void OFN(cart2sph_d)(int l, double* T) {
  real Tr[9 * 15];
  OFN(cart2sph)(l, Tr);
  for (int k = 0; k < (2 * l + 1) * NCART(l); ++k) T[k] = (double)Tr[k];
}
