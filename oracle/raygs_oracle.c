/*
 * raygs_oracle.c -- plain FP64 CPU oracle for ray-based Gaussian splatting (RayGS).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference leg load this library.  The CUDA renderer never calls it, and
 * the two share no code: no headers, no helpers, no constants.
 *
 * What it computes is the plain definition of the image, brute force over every pixel and
 * every primitive:
 *
 *   - Primitive activation (Sec. 3, "Scene representation"): Sigma = R S^2 R^T with R from
 *     a unit quaternion (here: by Hamilton products, R e_j = q (0,e_j) q*), S = diag(exp
 *     log-scale), prior opacity o = sigmoid(logit), all expressed in the camera frame.
 *   - Anti-aliasing (Sec. 5, Eq. mip): Sigma^ = Sigma + lambda I with the pixel-invariant
 *     lambda = sigma^2 * tau_bar^2 / (fx fy), tau_bar = |mu| (tau of the unit ray through the
 *     mean), and the opacity modulated by sqrt(|Sigma| c^2 / (|Sigma^| c^^2)).
 *   - Exact pixel-dependent anti-aliasing (Sec. 5 and its appendix derivation of P_MIP),
 *     camera mip = 2: per unit pixel ray x, Sigma^_x = Sigma + sigma_x^2 tau(x)^2 I with
 *     tau(x) the ray's maximum-density distance under Sigma and sigma_x^2 = sigma^2
 *     cos^3(theta) / (fx fy) the pixel's area at unit distance along the ray;
 *     omega = o m(x) exp(-D_ray(x; mu, Sigma^_x) / 2) with the modulation
 *     m(x) = sqrt(|Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x)), counted when
 *     omega >= p_min.  Camera-inside skip and kappa as for the plain primitive.
 *   - Support cut-off (Sec. 3, Eq. support): kappa = -2 log(p_min / o); a primitive with
 *     kappa <= 0 is skipped.
 *   - Camera-inside skip (Sec. 3.2, Eq. c): skip when c^2 = mu^T Sigma^-1 mu <= kappa.
 *   - Divergence (Sec. 3.2, Eq. Q_ray): tau = x^T Sigma^-1 mu / x^T Sigma^-1 x and
 *     D_ray = (tau x - mu)^T Sigma^-1 (tau x - mu), evaluated per pixel ray.
 *   - GS divergence (Sec. 3.1), selected by the configuration instead of D_ray:
 *     D_gs = (pi(x) - pi(mu))^T Sigma_pi^-1 (pi(x) - pi(mu)), Sigma_pi = J Sigma J^T with J
 *     the Jacobian of the pinhole projection at the mean, pi(x) the pixel centre.  There
 *     is no camera-inside skip and no Eq. mip term for it (a MIP camera is refused).
 *   - Rendered opacity (Sec. 3, Eq. rend_opacity): omega = o exp(-D/2); it counts only
 *     when D <= kappa (equivalently omega >= p_min).
 *   - Rendering equation (Sec. 3, Eq. rendering): front-to-back compositing over the
 *     primitives in ascending order of their centre's depth.
 *
 * Readings taken where the paper is silent:
 *   - only rays with tau > 0 count (the density maximum lies in front of the camera);
 *   - the near plane culls whole primitives (Sec. 4.1, "near plane clipping");
 *   - omega is clamped to alpha_max (0.99) and compositing stops before a primitive that
 *     would bring the transmittance below t_stop (1e-4); the background is black;
 *   - the depth order key is the float32 view-space depth of the mean, evaluated as the
 *     fused chain fmaf(R20, x, fmaf(R21, y, fmaf(R22, z, t2))) (the renderer's own
 *     precision, so that both sides take this integer decision identically); ties go to the
 *     lower primitive index;
 *   - colour: rgb = max(0, k_0 + sum_{l>=1} sum_m Y_lm(d) k_lm) with the real spherical
 *     harmonics without Condon-Shortley phase, d the unit vector from the camera centre to
 *     the mean in world space, k_0 stored directly as the base colour.
 *
 * The paper's vertex stage (Sec. 4.1 and App. A.1-A.3: the rotation R_{mu^<-v}, the
 * matrix Q, the quad orientation U_ray from the 2x2 eigen-problem Eq. optim2 and the quad
 * vertices Eq. V_ray) is written out below as well, in the paper's order and notation, for
 * the vertex-stage tests (quad containment, fragment identity, ...).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846

/* camera record: 20 doubles holding float32 values */
enum { CAM_FX = 0, CAM_FY, CAM_CX, CAM_CY, CAM_W, CAM_H, CAM_R = 6, CAM_T = 15,
       CAM_NEAR = 18, CAM_MIP = 19, CAM_LEN = 20 };
/* configuration: p_min, t_stop, alpha_max, mip sigma^2 (pixel units) */
/* CFG_DIV: 0 for the ray divergence D_ray (Eq. Q_ray), 1 for the GS divergence D_gs of
 * Sec. 3.1 (EWA: Mahalanobis distance in pixel space under Sigma_pi = J Sigma J^T, J the
 * Jacobian of the projection at the mean) */
enum { CFG_PMIN = 0, CFG_TSTOP, CFG_AMAX, CFG_MIPS2, CFG_DIV, CFG_LEN };

/* per-primitive output record of oracle_prepare (doubles) */
enum {
  OG_STATUS = 0,   /* 0 rendered, 1 near-plane cull, 2 kappa<=0, 3 c^2<=kappa, 4 non-finite */
  OG_KEY,          /* depth key (uint32 bits of the float32 depth) */
  OG_MU = 2,       /* camera-frame mean (3) */
  OG_C2 = 5, OG_KAPPA, OG_O,
  OG_RGB = 8,      /* colour (3) */
  OG_S = 11,       /* scales after the anti-aliasing term (3) */
  OG_RC = 14,      /* camera-frame rotation R_c (9, row-major) */
  OG_BORDER = 23,  /* 1 when a skip decision sits within FP64 rounding of its threshold */
  OG_LEN = 24
};

/* flags per pixel */
enum { FLAG_CUTOFF = 1, FLAG_STOP = 2, FLAG_BORDER = 4 };

/* ------------------------------------------------------------------ small helpers */

static void qmul(const double a[4], const double b[4], double r[4]) {
  /* Hamilton product, (w, x, y, z) */
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* Rotation matrix of a (not necessarily unit) quaternion: column j = q (0, e_j) q*. */
void oracle_quat_to_rot(const double qin[4], double R[9]) {
  double nrm = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double q[4] = {qin[0] / nrm, qin[1] / nrm, qin[2] / nrm, qin[3] / nrm};
  double qc[4] = {q[0], -q[1], -q[2], -q[3]};
  for (int j = 0; j < 3; ++j) {
    double e[4] = {0, 0, 0, 0}, t[4], r[4];
    e[1 + j] = 1.0;
    qmul(q, e, t);
    qmul(t, qc, r);
    for (int i = 0; i < 3; ++i) R[3 * i + j] = r[1 + i];
  }
}

static void matmul3(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

/* Associated Legendre function P_l^m(t), m >= 0, without the Condon-Shortley phase. */
static double legendre(int l, int m, double t, double st) {
  double pmm = 1.0;
  for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * st;
  if (l == m) return pmm;
  double pm1 = t * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pm1;
  double pl = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pl = ((2.0 * ll - 1.0) * t * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pm1;
    pm1 = pl;
  }
  return pl;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

/* Real spherical harmonics Y_lm(d), l <= degree, at index l*l + l + m. */
void oracle_sh_basis(int degree, const double d[3], double *Y) {
  double t = d[2];
  double st = sqrt(fmax(0.0, 1.0 - t * t));
  double phi = atan2(d[1], d[0]);
  for (int l = 0; l <= degree; ++l)
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * O_PI) * factorial(l - am) / factorial(l + am));
      double P = legendre(l, am, t, st);
      double y;
      if (m == 0) y = K * P;
      else if (m > 0) y = sqrt(2.0) * K * cos(m * phi) * P;
      else y = sqrt(2.0) * K * sin(am * phi) * P;
      Y[l * l + l + m] = y;
    }
}

/* Depth key: float32 bits of the fused chain fmaf(R20,x,fmaf(R21,y,fmaf(R22,z,t2))). */
uint32_t oracle_depth_key(const float r2[3], float t2, const float mu[3], float *z_out) {
  float z = fmaf(r2[0], mu[0], fmaf(r2[1], mu[1], fmaf(r2[2], mu[2], t2)));
  if (z_out) *z_out = z;
  uint32_t k;
  memcpy(&k, &z, 4);
  return k;
}

/* ------------------------------------------------------------ RayGS definitions */

/* Eq. Q_ray: tau(x) = x^T Si mu / x^T Si x, D = (tau x - mu)^T Si (tau x - mu). */
double oracle_D_ray(const double mu[3], const double Si[9], const double x[3], double *tau_out) {
  double Six[3], Simu[3];
  for (int i = 0; i < 3; ++i) {
    Six[i] = Si[3 * i] * x[0] + Si[3 * i + 1] * x[1] + Si[3 * i + 2] * x[2];
    Simu[i] = Si[3 * i] * mu[0] + Si[3 * i + 1] * mu[1] + Si[3 * i + 2] * mu[2];
  }
  double num = x[0] * Simu[0] + x[1] * Simu[1] + x[2] * Simu[2];
  double den = x[0] * Six[0] + x[1] * Six[1] + x[2] * Six[2];
  double tau = num / den;
  double r[3] = {tau * x[0] - mu[0], tau * x[1] - mu[1], tau * x[2] - mu[2]};
  double D = 0;
  for (int i = 0; i < 3; ++i)
    D += r[i] * (Si[3 * i] * r[0] + Si[3 * i + 1] * r[1] + Si[3 * i + 2] * r[2]);
  if (tau_out) *tau_out = tau;
  return D;
}

/* Support of one primitive over a pixel rectangle [x0, x0+w) x [y0, y0+h): out[j*w+i] = 1
 * when the ray through the centre of pixel (x0+i, y0+j) has tau > 0 and D <= kappa
 * (Eq. Q_ray and the cut-off of Sec. 3), else 0.  cam = (fx, fy, cx, cy). */
void oracle_support_mask(const double mu[3], const double Si[9], double kappa, const double cam[4], int x0, int y0,
                         int w, int h, unsigned char *out) {
  for (int j = 0; j < h; ++j)
    for (int i = 0; i < w; ++i) {
      const double x[3] = {((x0 + i) + 0.5 - cam[2]) / cam[0], ((y0 + j) + 0.5 - cam[3]) / cam[1], 1.0};
      double tau;
      const double D = oracle_D_ray(mu, Si, x, &tau);
      out[j * w + i] = (tau > 0.0 && D <= kappa) ? 1 : 0;
    }
}

/* App. A.1: R_{x,y} = 2 (x+y)(x+y)^T / |x+y|^2 - I (aligns y to x). */
static void rot_xy(const double x[3], const double y[3], double R[9]) {
  double a[3] = {x[0] + y[0], x[1] + y[1], x[2] + y[2]};
  double n2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = 2.0 * a[i] * a[j] / n2 - (i == j ? 1.0 : 0.0);
}

/* App. A.1: R_{mu^<-v} = R_{mu^,v} if mu^.v >= 0, else R_{mu^,-v} P, P = diag(-1,1,-1). */
void oracle_rot_align(const double muhat[3], double R[9]) {
  const double v[3] = {0, 0, 1}, mv[3] = {0, 0, -1};
  if (muhat[2] >= 0) {
    rot_xy(muhat, v, R);
  } else {
    double Rm[9];
    rot_xy(muhat, mv, Rm);
    for (int i = 0; i < 3; ++i) {
      R[3 * i + 0] = -Rm[3 * i + 0];
      R[3 * i + 1] = Rm[3 * i + 1];
      R[3 * i + 2] = -Rm[3 * i + 2];
    }
  }
}

/*
 * Sec. 4.1 vertex stage for a primitive with camera-frame mean mu, rotation Rc (row-major)
 * and scales s, at cut-off kappa (requires c^2 > kappa).  Output layout (doubles):
 *   [0:12)  V_ray, 4 vertices as columns: V[3*j + i] = coordinate i of vertex j
 *   [12:20) Z_ray (2x4, Z[2*j + i])
 *   [20:24) U_ray = (u0, u1) as columns: U[2*j + i]
 *   [24] c^2, [25] b, [26] a
 *   [27:36) Q (row-major), [36:45) R_{mu^<-v} (row-major), [45:48) mu^
 */
void oracle_quad(const double mu[3], const double Rc[9], const double s[3], double kappa,
                 double *out) {
  /* mu^ = S^-1 R^T mu / c */
  double m[3];
  for (int k = 0; k < 3; ++k)
    m[k] = (Rc[k] * mu[0] + Rc[3 + k] * mu[1] + Rc[6 + k] * mu[2]) / s[k];
  double c2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
  double c = sqrt(c2);
  double muhat[3] = {m[0] / c, m[1] / c, m[2] / c};
  double Ra[9];
  oracle_rot_align(muhat, Ra);
  /* Eq. invPhi: Q = R_p S R_{mu^<-v} */
  double RS[9], Q[9];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) RS[3 * i + k] = Rc[3 * i + k] * s[k];
  matmul3(RS, Ra, Q);
  /* Eq. optim2: B = Q_{:,0:2}^T Q_{:,0:2}; u1 = eigenvector of the largest eigenvalue */
  double B00 = 0, B01 = 0, B11 = 0;
  for (int i = 0; i < 3; ++i) {
    B00 += Q[3 * i] * Q[3 * i];
    B01 += Q[3 * i] * Q[3 * i + 1];
    B11 += Q[3 * i + 1] * Q[3 * i + 1];
  }
  double u1[2];
  if (B01 == 0.0) {
    u1[0] = B00 >= B11 ? 1.0 : 0.0;
    u1[1] = B00 >= B11 ? 0.0 : 1.0;
  } else {
    double half = 0.5 * (B00 - B11);
    double lam = 0.5 * (B00 + B11) + sqrt(half * half + B01 * B01);
    double va[2] = {lam - B11, B01}, vb[2] = {B01, lam - B00};
    double na = hypot(va[0], va[1]), nb = hypot(vb[0], vb[1]);
    if (na >= nb) { u1[0] = va[0] / na; u1[1] = va[1] / na; }
    else { u1[0] = vb[0] / nb; u1[1] = vb[1] / nb; }
  }
  double u0[2] = {-u1[1], u1[0]}; /* +90 degrees, counter-clockwise */
  /* Eq. rel2 and rel4: b = sqrt(1 - kappa/c^2), a = sqrt(kappa / (c^2 - kappa)) */
  double b = sqrt(1.0 - kappa / c2);
  double a = sqrt(kappa / (c2 - kappa));
  /* Eq. V_ray: Z = (sqrt(kappa)/b) O, T = [Q_{0:2} U, mu], V = T H(Z) */
  static const double O[2][4] = {{-1, -1, 1, 1}, {-1, 1, 1, -1}};
  double zs = sqrt(kappa) / b;
  double T01[3][2];
  for (int i = 0; i < 3; ++i) {
    T01[i][0] = Q[3 * i] * u0[0] + Q[3 * i + 1] * u0[1];
    T01[i][1] = Q[3 * i] * u1[0] + Q[3 * i + 1] * u1[1];
  }
  for (int j = 0; j < 4; ++j) {
    double z0 = zs * O[0][j], z1 = zs * O[1][j];
    out[12 + 2 * j] = z0;
    out[12 + 2 * j + 1] = z1;
    for (int i = 0; i < 3; ++i) out[3 * j + i] = T01[i][0] * z0 + T01[i][1] * z1 + mu[i];
  }
  out[20] = u0[0]; out[21] = u0[1]; out[22] = u1[0]; out[23] = u1[1];
  out[24] = c2; out[25] = b; out[26] = a;
  for (int i = 0; i < 9; ++i) { out[27 + i] = Q[i]; out[36 + i] = Ra[i]; }
  for (int i = 0; i < 3; ++i) out[45 + i] = muhat[i];
}

/* ------------------------------------------------------------ per-primitive setup */

typedef struct {
  int status, border;
  uint32_t key;
  int64_t index;
  double mu[3];    /* camera-frame mean */
  double W[9];     /* whitening map S^-1 R_c^T, row-major: Sigma^-1 = W^T W */
  double m[3];     /* W mu */
  double c2, kappa, o, rgb[3], s[3], Rc[9];
  double u[2], A[3]; /* GS: projected mean (pixels) and Sigma_pi^-1 = [[A0, A1], [A1, A2]] */
} prim;

static void prepare_one(int64_t i, const float *means, const float *log_scales,
                        const float *quats, const float *logits, const float *sh,
                        int sh_degree, const double *cam, const double *cfg, prim *g) {
  memset(g, 0, sizeof(*g));
  g->index = i;
  const float *mw = means + 3 * i;
  double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
  double ls[3] = {log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]};
  double logit = logits[i];
  int finite = isfinite(mw[0]) && isfinite(mw[1]) && isfinite(mw[2]) && isfinite(logit);
  for (int k = 0; k < 4; ++k) finite = finite && isfinite(q[k]);
  for (int k = 0; k < 3; ++k) finite = finite && isfinite(ls[k]);
  double qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!finite || !(qn > 0)) { g->status = 4; return; }

  float r2[3] = {(float)cam[CAM_R + 6], (float)cam[CAM_R + 7], (float)cam[CAM_R + 8]};
  float zf;
  g->key = oracle_depth_key(r2, (float)cam[CAM_T + 2], mw, &zf);
  if (!(zf > (float)cam[CAM_NEAR])) { g->status = 1; return; }

  const double *Rwc = cam + CAM_R, *twc = cam + CAM_T;
  for (int r = 0; r < 3; ++r)
    g->mu[r] = Rwc[3 * r] * (double)mw[0] + Rwc[3 * r + 1] * (double)mw[1] +
               Rwc[3 * r + 2] * (double)mw[2] + twc[r];
  double Rp[9];
  oracle_quat_to_rot(q, Rp);
  matmul3(Rwc, Rp, g->Rc);
  double s2[3];
  for (int k = 0; k < 3; ++k) { g->s[k] = exp(ls[k]); s2[k] = g->s[k] * g->s[k]; }
  double o = 1.0 / (1.0 + exp(-logit));
  double Rtmu[3];
  for (int k = 0; k < 3; ++k)
    Rtmu[k] = g->Rc[k] * g->mu[0] + g->Rc[3 + k] * g->mu[1] + g->Rc[6 + k] * g->mu[2];

  const int gs_div = (int)cfg[CFG_DIV] == 1;
  /* Rounding model of the two skip decisions below.  Two FP64 evaluations of this stage
   * (this one and a renderer's) differ mainly through the camera-frame mean, which may
   * carry a relative error up to E_MU; R_c^T mu then moves by up to E_MU |mu|_1 per axis,
   * and m_k = (R_c^T mu)_k / s_k by that over s_k (large for thin primitives seen from
   * near their plane). */
  const double E_MU = 1e-11;
  const double mu1 = fabs(g->mu[0]) + fabs(g->mu[1]) + fabs(g->mu[2]);
  double rel_o = 1e-12; /* relative rounding bound of the opacity */
  if ((int)cam[CAM_MIP] == 1) {
    /* Eq. mip with the pixel-invariant Sigma^ = Sigma + lambda I */
    double mu2 = g->mu[0] * g->mu[0] + g->mu[1] * g->mu[1] + g->mu[2] * g->mu[2];
    double lam = cfg[CFG_MIPS2] * mu2 / (cam[CAM_FX] * cam[CAM_FY]);
    double c2 = 0, c2h = 0, det = 1, deth = 1, e2 = 0, e2h = 0;
    for (int k = 0; k < 3; ++k) {
      double sh2 = s2[k] + lam;
      c2 += Rtmu[k] * Rtmu[k] / s2[k];
      c2h += Rtmu[k] * Rtmu[k] / sh2;
      e2 += 2.0 * fabs(Rtmu[k]) * E_MU * mu1 / s2[k];
      e2h += 2.0 * fabs(Rtmu[k]) * E_MU * mu1 / sh2;
      det *= s2[k];
      deth *= sh2;
      s2[k] = sh2;
      g->s[k] = sqrt(sh2);
    }
    o *= sqrt(det * c2 / (deth * c2h));
    rel_o += 0.5 * (e2 / c2 + e2h / c2h);
  }
  g->o = o;
  double pmin = cfg[CFG_PMIN];
  g->kappa = -2.0 * log(pmin / o);
  /* Eq. support: skip when kappa <= 0, i.e. o <= p_min */
  if (fabs(log(o / pmin)) <= rel_o) g->border = 1;

  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) g->W[3 * k + j] = g->Rc[3 * j + k] / g->s[k];
  for (int k = 0; k < 3; ++k) g->m[k] = Rtmu[k] / g->s[k];
  g->c2 = g->m[0] * g->m[0] + g->m[1] * g->m[1] + g->m[2] * g->m[2];
  double e_c2 = 1e-12 * g->c2 + 2.0 * rel_o; /* + the rounding of kappa */
  for (int k = 0; k < 3; ++k) e_c2 += 2.0 * fabs(g->m[k]) * E_MU * mu1 / g->s[k];
  if (gs_div) {
    /* Sec. 3.1: Sigma_pi = J Sigma J^T with J the Jacobian of pi(p) = (fx p_x / p_z + cx,
     * fy p_y / p_z + cy) at the camera-frame mean; Sigma = R_c S^2 R_c^T */
    double Sg[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double v = 0;
        for (int k = 0; k < 3; ++k) v += g->Rc[3 * a + k] * s2[k] * g->Rc[3 * b + k];
        Sg[3 * a + b] = v;
      }
    const double z = g->mu[2], fx = cam[CAM_FX], fy = cam[CAM_FY];
    const double J[6] = {fx / z, 0.0, -fx * g->mu[0] / (z * z), 0.0, fy / z, -fy * g->mu[1] / (z * z)};
    double P[4];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double v = 0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) v += J[3 * a + i] * Sg[3 * i + j] * J[3 * b + j];
        P[2 * a + b] = v;
      }
    const double det = P[0] * P[3] - P[1] * P[2];
    g->A[0] = P[3] / det;
    g->A[1] = -P[1] / det;
    g->A[2] = P[0] / det;
    g->u[0] = fx * g->mu[0] / z + cam[CAM_CX];
    g->u[1] = fy * g->mu[1] / z + cam[CAM_CY];
  }
  if (!(g->kappa > 0)) { g->status = 2; return; }
  if (!gs_div) {
    /* Sec. 3.2 Eq. c: skip when c^2 <= kappa */
    if (fabs(g->c2 - g->kappa) <= e_c2) g->border = 1;
    if (!(g->c2 > g->kappa)) { g->status = 3; return; }
  }

  /* colour: direction from the camera centre C = -R^T t to the world-frame mean */
  double C[3], d[3], dn = 0;
  for (int k = 0; k < 3; ++k)
    C[k] = -(Rwc[k] * twc[0] + Rwc[3 + k] * twc[1] + Rwc[6 + k] * twc[2]);
  for (int k = 0; k < 3; ++k) { d[k] = (double)mw[k] - C[k]; dn += d[k] * d[k]; }
  dn = sqrt(dn);
  for (int k = 0; k < 3; ++k) d[k] /= dn;
  int K = (sh_degree + 1) * (sh_degree + 1);
  double Y[16];
  oracle_sh_basis(sh_degree, d, Y);
  const float *f = sh + (int64_t)3 * K * i;
  for (int ch = 0; ch < 3; ++ch) {
    double v = f[ch];
    for (int k = 1; k < K; ++k) v += Y[k] * (double)f[3 * k + ch];
    g->rgb[ch] = v > 0 ? v : 0.0;
  }
}

/* The rendered opacity of primitive g at the pixel (px, py) with ray x, before the cut-off
 * and the clamp: *om = o m(x) exp(-D/2) and *D_out = D, with D = D_ray (Eq. Q_ray), D_gs
 * (Sec. 3.1) or the exact anti-aliased D_ray under Sigma^_x (Sec. 5; m(x) its modulation,
 * else m = 1).  Returns 0 when the pixel does not count (tau <= 0). */
static int pixel_weight(const prim *g, const double x[3], int px, int py, int mip_exact, int gs_div,
                        double sig2, double *D_out, double *om) {
  double D, mod = 1.0;
  if (mip_exact) {
    /* Sec. 5: unit ray xh, tau(xh) under Sigma, lambda = sigma_x^2 tau^2, then D_ray and
     * the modulation under Sigma^_x = Sigma + lambda I, both in Sigma's eigenframe
     * (Sigma = R_c diag(s^2) R_c^T, so Sigma^_x = R_c diag(s^2 + lambda) R_c^T). */
    const double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    const double xh[3] = {x[0] / xn, x[1] / xn, x[2] / xn};
    double a[3], b[3]; /* R_c^T xh and R_c^T mu */
    for (int j = 0; j < 3; ++j) {
      a[j] = g->Rc[j] * xh[0] + g->Rc[3 + j] * xh[1] + g->Rc[6 + j] * xh[2];
      b[j] = g->Rc[j] * g->mu[0] + g->Rc[3 + j] * g->mu[1] + g->Rc[6 + j] * g->mu[2];
    }
    double n0 = 0, d0 = 0;
    for (int j = 0; j < 3; ++j) {
      const double s2 = g->s[j] * g->s[j];
      n0 += b[j] * a[j] / s2;
      d0 += a[j] * a[j] / s2;
    }
    const double tau = n0 / d0;
    if (!(tau > 0)) return 0;
    const double cth = 1.0 / xn; /* cos of the ray's angle to the optical axis */
    /* lambda = sigma_x^2 tau(x)^2 with sigma_x^2 = sigma^2 cos^3(theta) / (fx fy), the
     * pixel's area at unit distance along the ray */
    const double lam = sig2 * cth * cth * cth * tau * tau;
    double n1 = 0, d1 = 0, ratio = 1;
    for (int j = 0; j < 3; ++j) {
      const double s2 = g->s[j] * g->s[j], sh2 = s2 + lam;
      n1 += b[j] * a[j] / sh2;
      d1 += a[j] * a[j] / sh2;
      ratio *= s2 / sh2;
    }
    const double tauh = n1 / d1;
    if (!(tauh > 0)) return 0;
    D = 0; /* (tauh xh - mu)^T Sigma^_x^-1 (tauh xh - mu) */
    for (int j = 0; j < 3; ++j) {
      const double r = tauh * a[j] - b[j];
      D += r * r / (g->s[j] * g->s[j] + lam);
    }
    /* modulation sqrt(|Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x)):
     * ratio = |Sigma| / |Sigma^_x|, d0 = x^T Sigma^-1 x, d1 = x^T Sigma^_x^-1 x (unit x) */
    mod = sqrt(ratio * d0 / d1);
  } else if (gs_div) {
    /* Sec. 3.1: (pi(x) - pi(mu))^T Sigma_pi^-1 (pi(x) - pi(mu)), pi(x) the pixel centre */
    const double dx = (px + 0.5) - g->u[0], dy = (py + 0.5) - g->u[1];
    D = g->A[0] * dx * dx + 2.0 * g->A[1] * dx * dy + g->A[2] * dy * dy;
  } else {
    double w[3];
    for (int r = 0; r < 3; ++r) w[r] = g->W[3 * r] * x[0] + g->W[3 * r + 1] * x[1] + g->W[3 * r + 2] * x[2];
    double num = g->m[0] * w[0] + g->m[1] * w[1] + g->m[2] * w[2]; /* x^T Si mu */
    double den = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];          /* x^T Si x  */
    double tau = num / den;
    if (!(tau > 0)) return 0;
    double r0 = tau * w[0] - g->m[0], r1 = tau * w[1] - g->m[1], r2 = tau * w[2] - g->m[2];
    D = r0 * r0 + r1 * r1 + r2 * r2;
  }
  *D_out = D;
  *om = g->o * mod * exp(-0.5 * D);
  return 1;
}

static int cmp_prim(const void *pa, const void *pb) {
  const prim *a = *(const prim *const *)pa, *b = *(const prim *const *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->index < b->index ? -1 : (a->index > b->index ? 1 : 0);
}

/* Per-primitive quantities for one camera (out: n x OG_LEN doubles). */
int oracle_prepare(int64_t n, const float *means, const float *log_scales, const float *quats,
                   const float *logits, const float *sh, int sh_degree, const double *cam,
                   const double *cfg, double *out) {
  if (n < 0 || sh_degree < 0 || sh_degree > 3) return 1;
  if ((int)cfg[CFG_DIV] == 1 && (int)cam[CAM_MIP]) return 4; /* Eq. mip is a RayGS term */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    prim g;
    prepare_one(i, means, log_scales, quats, logits, sh, sh_degree, cam, cfg, &g);
    double *o = out + OG_LEN * i;
    memset(o, 0, sizeof(double) * OG_LEN);
    o[OG_STATUS] = g.status;
    o[OG_KEY] = (double)g.key;
    for (int k = 0; k < 3; ++k) {
      o[OG_MU + k] = g.mu[k];
      o[OG_RGB + k] = g.rgb[k];
      o[OG_S + k] = g.s[k];
    }
    o[OG_C2] = g.c2;
    o[OG_KAPPA] = g.kappa;
    o[OG_O] = g.o;
    for (int k = 0; k < 9; ++k) o[OG_RC + k] = g.Rc[k];
    o[OG_BORDER] = g.border;
  }
  return 0;
}

/*
 * Render pixels of one camera.  pix: n_pix (x, y) pairs, or NULL for the whole image in
 * row-major order (then n_pix must equal W*H).  Outputs per pixel: rgb (3 doubles), final
 * transmittance, number of composited primitives, flags (cut-off / stop / border bands) and
 * a 64-bit signature of the composited primitive indices (may be NULL).
 */
int oracle_render(int64_t n, const float *means, const float *log_scales, const float *quats,
                  const float *logits, const float *sh, int sh_degree, const double *cam,
                  const double *cfg, int64_t n_pix, const int32_t *pix, double *rgb,
                  double *Tout, int32_t *ncontrib, int32_t *flags, uint64_t *sig,
                  int n_threads) {
  if (n < 0 || sh_degree < 0 || sh_degree > 3) return 1;
  if ((int)cfg[CFG_DIV] == 1 && (int)cam[CAM_MIP]) return 4; /* Eq. mip is a RayGS term */
  int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
  if (!pix && n_pix != (int64_t)W * H) return 2;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
  prim *gs = (prim *)malloc(sizeof(prim) * (n > 0 ? n : 1));
  if (!gs) return 3;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    prepare_one(i, means, log_scales, quats, logits, sh, sh_degree, cam, cfg, gs + i);
  int64_t nv = 0, nb = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (gs[i].status == 0) ++nv;
    if (gs[i].border && gs[i].status != 1 && gs[i].status != 4) ++nb;
  }
  prim **order = (prim **)malloc(sizeof(prim *) * (nv > 0 ? nv : 1));
  prim **border = (prim **)malloc(sizeof(prim *) * (nb > 0 ? nb : 1));
  if (!order || !border) { free(gs); free(order); free(border); return 3; }
  nv = nb = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (gs[i].status == 0) order[nv++] = gs + i;
    if (gs[i].border && gs[i].status != 1 && gs[i].status != 4) border[nb++] = gs + i;
  }
  qsort(order, (size_t)nv, sizeof(prim *), cmp_prim);

  const double fx = cam[CAM_FX], fy = cam[CAM_FY], cx = cam[CAM_CX], cy = cam[CAM_CY];
  const double pmin = cfg[CFG_PMIN], tstop = cfg[CFG_TSTOP], amax = cfg[CFG_AMAX];
  const int gs_div = (int)cfg[CFG_DIV] == 1;
  const int mip_exact = (int)cam[CAM_MIP] == 2;
  const double sig2 = cfg[CFG_MIPS2] / (fx * fy); /* sigma^2 per unit distance on the axis */

#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t p = 0; p < n_pix; ++p) {
    int px = pix ? pix[2 * p] : (int)(p % W);
    int py = pix ? pix[2 * p + 1] : (int)(p / W);
    double x[3] = {(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0};
    double C[3] = {0, 0, 0}, T = 1.0;
    int32_t cnt = 0, fl = 0;
    uint64_t h = 1469598103934665603ull;
    for (int64_t k = 0; k < nv; ++k) {
      const prim *g = order[k];
      double D, om;
      if (!pixel_weight(g, x, px, py, mip_exact, gs_div, sig2, &D, &om)) continue;
      if (fabs(om - pmin) <= 1e-6) fl |= FLAG_CUTOFF;
      if (mip_exact ? !(om >= pmin) : !(D <= g->kappa)) continue;
      if (om > amax) om = amax;
      double Tn = T * (1.0 - om);
      if (fabs(Tn - tstop) <= 1e-4 * tstop) fl |= FLAG_STOP;
      if (Tn < tstop) break;
      for (int ch = 0; ch < 3; ++ch) C[ch] += om * T * g->rgb[ch];
      T = Tn;
      ++cnt;
      h = (h ^ (uint64_t)(g->index + 1)) * 1099511628211ull;
    }
    /* a primitive whose skip decision sits within rounding of its threshold: the pixels it
     * would reach (omega >= p_min / 2) */
    for (int64_t k = 0; k < nb; ++k) {
      double D, om;
      if (pixel_weight(border[k], x, px, py, mip_exact, gs_div, sig2, &D, &om) && om >= 0.5 * pmin) {
        fl |= FLAG_BORDER;
        break;
      }
    }
    for (int ch = 0; ch < 3; ++ch) rgb[3 * p + ch] = C[ch];
    Tout[p] = T;
    if (ncontrib) ncontrib[p] = cnt;
    if (flags) flags[p] = fl;
    if (sig) sig[p] = h;
  }
  free(order);
  free(border);
  free(gs);
  return 0;
}
