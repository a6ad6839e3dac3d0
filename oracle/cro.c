/*
 * cro.c -- FP64 CPU oracle (test infrastructure only; see cro.h).
 *
 * Plain, single-threaded C99 written from the paper's equations, in the
 * paper's order and notation.  No blocking, fusion or reordering: one function
 * per equation, composed in cro_eval() the way Sec. 2-3 and App. A define the
 * cost.  It shares nothing with the CUDA library.
 */
#include "cro.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small 3x4 / 3-vector helpers (row-major 3x4: [R | p])                      */
/* ------------------------------------------------------------------------ */

static void tf_identity(double* T) {
  memset(T, 0, 12 * sizeof(double));
  T[0] = T[5] = T[10] = 1.0;
}

/* C = A * B for homogeneous 3x4 transforms */
static void tf_mul(const double* A, const double* B, double* C) {
  double out[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[r * 4 + k] * B[k * 4 + c];
      if (c == 3) s += A[r * 4 + 3];
      out[r * 4 + c] = s;
    }
  }
  memcpy(C, out, sizeof(out));
}

/* y = T * x (point) */
static void tf_point(const double* T, const double* x, double* y) {
  double o[3];
  for (int r = 0; r < 3; ++r)
    o[r] = T[r * 4 + 0] * x[0] + T[r * 4 + 1] * x[1] + T[r * 4 + 2] * x[2] + T[r * 4 + 3];
  memcpy(y, o, sizeof(o));
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double* a, const double* b, double* c) {
  double o[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  memcpy(c, o, sizeof(o));
}

static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static double dmin(double a, double b) { return a < b ? a : b; }

/* rotation matrix (row-major 3x3) of a unit quaternion w, x, y, z */
static void quat_to_rot(const double* q_in, double* R) {
  double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void note_margin(double* margin, double v) {
  if (margin && fabs(v) < *margin) *margin = fabs(v);
}

/* ------------------------------------------------------------------------ */
/* parameters: values stated in App. A.1-A.3, App. B.3 "cuRobo Parameters" and */
/* Sec. 7.3 "Line Search"; unstated ones take the readings listed per field.   */
/* ------------------------------------------------------------------------ */

void cro_params_default(cro_params* p) {
  memset(p, 0, sizeof(*p));
  p->w_goal_pos = 2000.0;   /* alpha_0, App. A.1 */
  p->w_goal_rot = 350.0;    /* alpha_1 */
  p->k_goal_pos = 100.0;    /* alpha_2 */
  p->k_goal_rot = 100.0;    /* alpha_3 */
  p->w_coll = 5000.0;       /* beta_2: soft-constraint weight 5000, App. B.3 */
  p->w_self = 5000.0;       /* beta_1 */
  p->w_bound = 5000.0;
  p->w_acc = 5000.0;        /* alpha_8, App. A.2 */
  p->w_jerk = 1.0;          /* alpha_9 */
  p->w_vel = 5000.0;        /* alpha_6 (only with CRO_VEL_COST; the set Q is not defined) */
  p->k_vel = 50.0;          /* alpha_7 */
  p->eta = 0.025;           /* 2.5 cm activation distance, App. B.3 */
  p->eta_bound = 0.1;       /* eta_2, App. A.3 */
  p->dt = 0.05;
  p->sweep_steps = 4;       /* unstated; reading */
  p->history = 6;
  p->n_alpha = 4;           /* Sec. 7.3: 0.01, 0.3, 0.7, 1.0 */
  p->alpha[0] = 0.01; p->alpha[1] = 0.3; p->alpha[2] = 0.7; p->alpha[3] = 1.0;
  p->armijo_c1 = 1e-4;      /* unstated (garbled in Alg. 1); textbook value */
  p->wolfe_c2 = 0.9;
  p->flags = CRO_SWEPT | CRO_SPEED | CRO_SELF | CRO_WOLFE;
  p->w_cspace = 5000.0;     /* alpha_4, App. A.1 (Eq. 15) */
  p->k_cspace = 50.0;       /* alpha_5 */
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 forward kinematics; App. E.1 Table "Joint Transformation matrices" */
/* ------------------------------------------------------------------------ */

/* Full link transformation F * J(theta) for a revolute joint about x, y or z:
 * the table's right-hand column, written as F times the joint rotation. */
static void joint_link_transform(const double* F, int axis, double theta, double* out) {
  double c = cos(theta), s = sin(theta);
  double J[12];
  tf_identity(J);
  if (axis == 0) {          /* Revolute X */
    J[5] = c; J[6] = -s; J[9] = s; J[10] = c;
  } else if (axis == 1) {   /* Revolute Y */
    J[0] = c; J[2] = s; J[8] = -s; J[10] = c;
  } else {                  /* Revolute Z */
    J[0] = c; J[1] = -s; J[4] = s; J[5] = c;
  }
  tf_mul(F, J, out);
}

void cro_fk(const cro_robot* rb, const double* theta, double* link_tf, double* spheres,
            double* ee) {
  double T[CRO_MAX_DOF][12];
  double prev[12];
  tf_identity(prev);
  for (int j = 0; j < rb->dof; ++j) {
    double A[12];
    joint_link_transform(rb->fixed_tf + 12 * j, rb->axis[j], theta[j], A);
    tf_mul(prev, A, T[j]);          /* T_j = T_{j-1} F_j J_j(theta_j) */
    memcpy(prev, T[j], sizeof(prev));
  }
  if (link_tf) memcpy(link_tf, T, (size_t)rb->dof * 12 * sizeof(double));
  if (ee) tf_mul(T[rb->dof - 1], rb->fixed_tf + 12 * rb->dof, ee);
  if (spheres) {
    for (int i = 0; i < rb->n_spheres; ++i) {
      tf_point(T[rb->sphere_link[i]], rb->spheres + 4 * i, spheres + 4 * i);
      spheres[4 * i + 3] = rb->spheres[4 * i + 3];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5 oriented bounding box: point signed distance                      */
/* ------------------------------------------------------------------------ */

/* Textbook box SDF in the box frame: positive outside (Euclidean distance to
 * the surface), minus the smallest face gap inside.  Gradient in the box
 * frame; inside, the face of the largest q wins, lowest axis on ties,
 * sign(0) := +1.  `face_gap` receives, for a point inside, the gap between the
 * two largest q (where the gradient switches face), else DBL_MAX. */
static double box_sdf_local(const double* u, const double* h, double* grad_u, double* face_gap) {
  double q[3], qp[3];
  for (int a = 0; a < 3; ++a) {
    q[a] = fabs(u[a]) - h[a];
    qp[a] = q[a] > 0.0 ? q[a] : 0.0;
  }
  double outside = norm3(qp);
  int amax = 0;
  for (int a = 1; a < 3; ++a)
    if (q[a] > q[amax]) amax = a;
  double maxq = q[amax];
  if (face_gap) {
    double second = -DBL_MAX;
    for (int a = 0; a < 3; ++a)
      if (a != amax && q[a] > second) second = q[a];
    *face_gap = outside > 0.0 ? DBL_MAX : maxq - second;
  }
  double phi = outside + dmin(maxq, 0.0);
  if (grad_u) {
    if (outside > 0.0) {
      for (int a = 0; a < 3; ++a) grad_u[a] = (u[a] >= 0.0 ? 1.0 : -1.0) * qp[a] / outside;
    } else {
      grad_u[0] = grad_u[1] = grad_u[2] = 0.0;
      grad_u[amax] = u[amax] >= 0.0 ? 1.0 : -1.0;
    }
  }
  return phi;
}

static double box_sdf(const double* pose7, const double* half_ext, const double* x, double* grad,
                      double* face_gap) {
  double R[9];
  quat_to_rot(pose7 + 3, R);
  double dx[3] = {x[0] - pose7[0], x[1] - pose7[1], x[2] - pose7[2]};
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = R[0 * 3 + a] * dx[0] + R[1 * 3 + a] * dx[1] + R[2 * 3 + a] * dx[2];
  double gu[3];
  double phi = box_sdf_local(u, half_ext, grad ? gu : NULL, face_gap);
  if (grad) {
    for (int r = 0; r < 3; ++r) grad[r] = R[r * 3 + 0] * gu[0] + R[r * 3 + 1] * gu[1] + R[r * 3 + 2] * gu[2];
  }
  return phi;
}

double cro_box_sdf(const double* pose7, const double* half_ext, const double* x, double* grad) {
  return box_sdf(pose7, half_ext, x, grad, NULL);
}

/* ------------------------------------------------------------------------ */
/* Eq. 10: smoothed collision distance of a penetration depth d               */
/* ------------------------------------------------------------------------ */

double cro_smooth_distance(double d, double eta, double* slope) {
  if (d > 0.0) {
    if (slope) *slope = 1.0;
    return d + 0.5 * eta;
  }
  if (d > -eta) {
    if (slope) *slope = (d + eta) / eta;
    return 0.5 / eta * (d + eta) * (d + eta);
  }
  if (slope) *slope = 0.0;
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 17: bound cost with activation eta_2                                   */
/* ------------------------------------------------------------------------ */

double cro_bound_cost(double q, double lo, double hi, double eta2, double* slope) {
  double c = 0.0, s = 0.0;
  if (q < lo) {
    c = lo - q + 0.5 * eta2;
    s = -1.0;
  } else if (q < lo + eta2) {
    c = 0.5 / eta2 * (lo - q + eta2) * (lo - q + eta2);
    s = -(lo - q + eta2) / eta2;
  } else if (q > hi) {
    c = q - hi + 0.5 * eta2;
    s = 1.0;
  } else if (q > hi - eta2) {
    c = 0.5 / eta2 * (q - hi + eta2) * (q - hi + eta2);
    s = (q - hi + eta2) / eta2;
  }
  if (slope) *slope = s;
  return c;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 continuous collision checking, for one sphere and one box         */
/* ------------------------------------------------------------------------ */

/* Penetration of the sphere (radius r) at point p into the box: r - phi(p);
 * gradient d pen / d p = -grad phi. */
static double penetration(const double* pose7, const double* h, double r, const double* p,
                          double* gpen, double* margin) {
  double g[3], gap;
  double phi = box_sdf(pose7, h, p, g, &gap);
  note_margin(margin, gap);
  if (gpen) {
    gpen[0] = -g[0]; gpen[1] = -g[1]; gpen[2] = -g[2];
  }
  return r - phi;
}

/* Reading of Sec. 3.4 / Fig. "sweep collision": check the waypoint x1 first;
 * if it is in collision (within eta of the box), add its smoothed distance and
 * move on by the inflated radius rhat = r + eta; otherwise move by the
 * sphere's signed distance to the box, phi - r (Sec. 3: the sphere distance is
 * the centre's distance minus the radius), which is at least eta there.
 * March from x1 toward each neighbour, at most `steps` samples, stopping at
 * the midpoint (half the distance to the neighbour).  Every sample in
 * collision adds its smoothed distance and moves on by rhat; every other
 * sample moves on by its sphere distance.  The gradient of every sample is
 * credited to the waypoint's own sphere (d sample / d x1 := I). */
double cro_sweep_box(const double* pose7, const double* half_ext, double r, const double* x0,
                     const double* x1, const double* x2, double eta, int32_t steps, double* g1,
                     double* margin) {
  double rhat = r + eta;
  double S = 0.0;
  double G[3] = {0, 0, 0};
  double gpen[3], slope;

  double pen1 = penetration(pose7, half_ext, r, x1, gpen, margin);
  note_margin(margin, pen1 + eta);
  double u0;
  if (pen1 > -eta) {
    S += cro_smooth_distance(pen1, eta, &slope);
    for (int a = 0; a < 3; ++a) G[a] += slope * gpen[a];
    u0 = rhat;
  } else {
    u0 = -pen1; /* phi(x1) - r */
  }

  const double* nb[2] = {x0, x2};
  for (int side = 0; side < 2; ++side) {
    const double* xn = nb[side];
    if (!xn) continue;
    double diff[3] = {xn[0] - x1[0], xn[1] - x1[1], xn[2] - x1[2]};
    double dist = norm3(diff);
    double L = 0.5 * dist;
    if (L == 0.0) continue;
    double dir[3] = {diff[0] / dist, diff[1] / dist, diff[2] / dist};
    double u = u0;
    for (int j = 0; j < steps; ++j) {
      double p[3] = {x1[0] + u * dir[0], x1[1] + u * dir[1], x1[2] + u * dir[2]};
      double mface = DBL_MAX;
      double pen = penetration(pose7, half_ext, r, p, gpen, &mface);
      /* Margin bookkeeping only.  The stop test u >= L can change the result
       * only when the sample at u is in collision: a sample out of collision
       * adds nothing, and the next step (at least eta) passes L anyway.  So
       * its distance from deciding anything is the larger of |u - L| and the
       * sample's distance from the activation threshold. */
      note_margin(margin, fmax(fabs(u - L), -eta - pen));
      if (u >= L) break;
      note_margin(margin, mface);
      note_margin(margin, pen + eta);
      if (pen > -eta) {
        S += cro_smooth_distance(pen, eta, &slope);
        for (int a = 0; a < 3; ++a) G[a] += slope * gpen[a];
        u += rhat;
      } else {
        u += -pen; /* phi(p) - r */
      }
    }
  }
  if (g1) memcpy(g1, G, sizeof(G));
  return S;
}

/* ------------------------------------------------------------------------ */
/* Eq. 9: self-collision, largest penetration over the pair set S             */
/* ------------------------------------------------------------------------ */

double cro_self_penetration(const cro_robot* rb, const double* X, int32_t* argmax,
                            double* grad_x) {
  double best = 0.0;
  int32_t arg = -1;
  for (int32_t p = 0; p < rb->n_pairs; ++p) {
    int i = rb->pairs[2 * p], j = rb->pairs[2 * p + 1];
    double ri = X[4 * i + 3], rj = X[4 * j + 3];
    if (ri <= 0.0 || rj <= 0.0) continue;
    double d[3] = {X[4 * i] - X[4 * j], X[4 * i + 1] - X[4 * j + 1], X[4 * i + 2] - X[4 * j + 2]};
    double pen = ri + rj - norm3(d);
    if (pen > best) {      /* strict: the first pair in list order wins ties */
      best = pen;
      arg = p;
    }
  }
  if (argmax) *argmax = arg;
  if (grad_x) {
    memset(grad_x, 0, (size_t)rb->n_spheres * 3 * sizeof(double));
    if (arg >= 0) {
      int i = rb->pairs[2 * arg], j = rb->pairs[2 * arg + 1];
      double d[3] = {X[4 * i] - X[4 * j], X[4 * i + 1] - X[4 * j + 1], X[4 * i + 2] - X[4 * j + 2]};
      double n = norm3(d);
      if (n > 0.0) {
        for (int a = 0; a < 3; ++a) {
          grad_x[3 * i + a] -= d[a] / n;
          grad_x[3 * j + a] += d[a] / n;
        }
      }
    }
  }
  return best;
}

/* gap between the best and the runner-up penetration (argmax stability) */
static double self_argmax_gap(const cro_robot* rb, const double* X) {
  double best = 0.0, second = 0.0;
  for (int32_t p = 0; p < rb->n_pairs; ++p) {
    int i = rb->pairs[2 * p], j = rb->pairs[2 * p + 1];
    double ri = X[4 * i + 3], rj = X[4 * j + 3];
    if (ri <= 0.0 || rj <= 0.0) continue;
    double d[3] = {X[4 * i] - X[4 * j], X[4 * i + 1] - X[4 * j + 1], X[4 * i + 2] - X[4 * j + 2]};
    double pen = ri + rj - norm3(d);
    if (pen > best) {
      second = best;
      best = pen;
    } else if (pen > second) {
      second = pen;
    }
  }
  return best > 0.0 ? best - second : DBL_MAX;
}

/* ------------------------------------------------------------------------ */
/* App. A.5 five-point stencils over the padded sequence of App. A.2           */
/* ------------------------------------------------------------------------ */

/* Implicit boundary states (App. A.2, Table "trajectory profiles", last row):
 * three copies of the start state before theta_1 and two more copies of
 * theta_H after it. */
static const double* ext_at(int32_t H, int32_t dof, const double* q0, const double* theta, int e) {
  if (e <= 2) return q0;
  if (e >= H + 2) return theta + (size_t)(H - 1) * dof;
  return theta + (size_t)(e - 3) * dof;
}

void cro_stencil(int32_t H, int32_t dof, const double* q0, const double* theta, double dt,
                 double* vel, double* acc, double* jerk) {
  for (int e = 2; e <= H + 2; ++e) {
    const double* qm2 = ext_at(H, dof, q0, theta, e - 2);
    const double* qm1 = ext_at(H, dof, q0, theta, e - 1);
    const double* q00 = ext_at(H, dof, q0, theta, e);
    const double* qp1 = ext_at(H, dof, q0, theta, e + 1);
    const double* qp2 = ext_at(H, dof, q0, theta, e + 2);
    int k = e - 2;
    for (int j = 0; j < dof; ++j) {
      vel[k * dof + j] = (qm2[j] - 8.0 * qm1[j] + 8.0 * qp1[j] - qp2[j]) / (12.0 * dt);
      acc[k * dof + j] = (-qm2[j] + 16.0 * qm1[j] - 30.0 * q00[j] + 16.0 * qp1[j] - qp2[j]) / (12.0 * dt * dt);
      jerk[k * dof + j] = (-qm2[j] + 2.0 * qm1[j] - 2.0 * qp1[j] + qp2[j]) / (2.0 * dt * dt * dt);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. 14: pose-reaching cost                                                 */
/* ------------------------------------------------------------------------ */

/* log cosh(x) = |x| + log(1 + exp(-2|x|)) - log 2, stable for large |x| */
static double logcosh(double x) {
  double a = fabs(x);
  return a + log1p(exp(-2.0 * a)) - log(2.0);
}

/* Orientation distance: 1 - (q_g . q)^2 = (3 - tr(R_g^T R)) / 4, which is
 * sign-invariant in the quaternions (reading of the similarity q_g^T q_T). */
double cro_goal_cost(const cro_params* prm, const double* ee, const double* goal7, double* dp,
                     double* dR) {
  double Rg[9];
  quat_to_rot(goal7 + 3, Rg);
  double e[3] = {ee[3] - goal7[0], ee[7] - goal7[1], ee[11] - goal7[2]};
  double r = norm3(e);
  double tr = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) tr += Rg[a * 3 + b] * ee[a * 4 + b];
  double dq = (3.0 - tr) / 4.0;
  double c = prm->w_goal_pos * logcosh(prm->k_goal_pos * r) +
             prm->w_goal_rot * logcosh(prm->k_goal_rot * dq);
  if (dp) {
    /* d/dp of alpha_0 logcosh(alpha_2 r) = alpha_0 alpha_2 tanh(alpha_2 r) e / r,
     * whose limit at r -> 0 is alpha_0 alpha_2^2 e */
    double f = r > 1e-300 ? prm->w_goal_pos * prm->k_goal_pos * tanh(prm->k_goal_pos * r) / r
                          : prm->w_goal_pos * prm->k_goal_pos * prm->k_goal_pos;
    for (int a = 0; a < 3; ++a) dp[a] = f * e[a];
  }
  if (dR) {
    double f = prm->w_goal_rot * prm->k_goal_rot * tanh(prm->k_goal_rot * dq) * (-0.25);
    for (int a = 0; a < 9; ++a) dR[a] = f * Rg[a];
  }
  return c;
}

/* ------------------------------------------------------------------------ */
/* the whole evaluation of one problem (Eq. 1 with soft constraints)           */
/* ------------------------------------------------------------------------ */

typedef struct {
  double pose[7];
  double h[3];
} box_t;

/* Backward kinematics (Sec. 3.1, App. E.1 Table "Gradient for different joint
 * types"): revolute joint j moves a point x of a link at or after j by
 * a_j x (x - o_j), and rotates an attached frame R by [a_j]_x R.  a_j is the
 * joint axis in the world and o_j the joint origin, both read from T_j. */
static void backward_state(const cro_robot* rb, const double* LT, const double* X,
                           const double* gx, const double* ee, const double* dp, const double* dR,
                           double* gtheta) {
  for (int j = 0; j < rb->dof; ++j) {
    const double* T = LT + 12 * j;
    double a[3] = {T[0 * 4 + rb->axis[j]], T[1 * 4 + rb->axis[j]], T[2 * 4 + rb->axis[j]]};
    double o[3] = {T[3], T[7], T[11]};
    double g = 0.0;
    for (int i = 0; i < rb->n_spheres; ++i) {
      if (rb->sphere_link[i] < j) continue;
      double rel[3] = {X[4 * i] - o[0], X[4 * i + 1] - o[1], X[4 * i + 2] - o[2]};
      double col[3];
      cross3(a, rel, col);
      g += dot3(gx + 3 * i, col);
    }
    if (ee) {
      double rel[3] = {ee[3] - o[0], ee[7] - o[1], ee[11] - o[2]};
      double col[3];
      cross3(a, rel, col);
      g += dot3(dp, col);
      /* <dR, [a]_x R> summed over the three columns of R */
      for (int c = 0; c < 3; ++c) {
        double Rc[3] = {ee[0 * 4 + c], ee[1 * 4 + c], ee[2 * 4 + c]};
        double aRc[3];
        cross3(a, Rc, aRc);
        g += dR[0 * 3 + c] * aRc[0] + dR[1 * 3 + c] * aRc[1] + dR[2 * 3 + c] * aRc[2];
      }
    }
    gtheta[j] = g;
  }
}

static void eval_one(const cro_robot* rb, const box_t* boxes, int32_t K, const double* q_start,
                     const double* goal7, const double* goal_q, const cro_params* prm, int32_t H,
                     const double* theta,
                     double* cost, double* grad, uint8_t* cfree, double* terms, double* margin,
                     double* st_terms, double* st_margin, double* st_clear) {
  const int D = rb->dof, M = rb->n_spheres;
  const int ik = (prm->flags & CRO_IK_MODE) != 0;
  const int swept = !ik && (prm->flags & CRO_SWEPT);
  const int speed = !ik && (prm->flags & CRO_SPEED);
  double term[CRO_N_TERMS] = {0, 0, 0, 0, 0};
  double mg = DBL_MAX;
  int free_ok = 1;
  /* per-state bookkeeping (world and self cost of each state, the margin of
   * the decisions that set its cost and gradient, its smallest clearance) */
  double* sw = (double*)calloc((size_t)H, sizeof(double));
  double* ss = (double*)calloc((size_t)H, sizeof(double));
  double* smg = (double*)malloc((size_t)H * sizeof(double));
  double* scl = (double*)malloc((size_t)H * sizeof(double));
  for (int t = 0; t < H; ++t) smg[t] = scl[t] = DBL_MAX;

  /* forward kinematics of the start state (slot 0) and of theta_1..theta_H */
  double* LT = (double*)calloc((size_t)(H + 1) * D * 12, sizeof(double));
  double* X = (double*)calloc((size_t)(H + 1) * M * 4, sizeof(double));
  double* GX = (double*)calloc((size_t)(H + 1) * M * 3, sizeof(double));
  double ee[12];
  cro_fk(rb, q_start, LT, X, NULL);
  for (int t = 1; t <= H; ++t)
    cro_fk(rb, theta + (size_t)(t - 1) * D, LT + (size_t)t * D * 12, X + (size_t)t * M * 4,
           t == H ? ee : NULL);

  /* Eq. 11 world term: beta_2 speed(S_{t-1,t,t+1}) smooth(sweep(S_{t-1,t,t+1})) */
  for (int t = 1; t <= H; ++t) {
    int tp = t < H ? t + 1 : H; /* x_{H+1} := x_H */
    for (int i = 0; i < M; ++i) {
      double r = X[((size_t)t * M + i) * 4 + 3];
      if (r < 0.0) continue; /* negative radius disables a sphere */
      const double* x1 = X + ((size_t)t * M + i) * 4;
      const double* x0 = X + ((size_t)(t - 1) * M + i) * 4;
      const double* x2 = X + ((size_t)tp * M + i) * 4;
      double Ssum = 0.0, gS[3] = {0, 0, 0};
      for (int k = 0; k < K; ++k) {
        double g1[3];
        Ssum += cro_sweep_box(boxes[k].pose, boxes[k].h, r, swept ? x0 : NULL, x1,
                              swept ? x2 : NULL, prm->eta, prm->sweep_steps, g1, &smg[t - 1]);
        for (int a = 0; a < 3; ++a) gS[a] += g1[a];
        /* validity flag: discrete clearance phi - r > 0 at every waypoint */
        double clear = cro_box_sdf(boxes[k].pose, boxes[k].h, x1, NULL) - r;
        if (clear < scl[t - 1]) scl[t - 1] = clear;
        if (!(clear > 0.0)) free_ok = 0;
      }
      double v = 1.0, dv[3] = {0, 0, 0};
      if (speed) {
        double diff[3] = {x2[0] - x0[0], x2[1] - x0[1], x2[2] - x0[2]};
        double n = norm3(diff);
        v = n / (2.0 * prm->dt);
        if (n > 0.0)
          for (int a = 0; a < 3; ++a) dv[a] = diff[a] / (n * 2.0 * prm->dt);
      }
      term[0] += prm->w_coll * v * Ssum;
      sw[t - 1] += prm->w_coll * v * Ssum;
      double* gx1 = GX + ((size_t)t * M + i) * 3;
      for (int a = 0; a < 3; ++a) gx1[a] += prm->w_coll * v * gS[a];
      if (speed && Ssum != 0.0) {
        /* product rule through speed = |x_{t+1} - x_{t-1}| / 2dt */
        double* gxp = GX + ((size_t)tp * M + i) * 3;
        double* gxm = GX + ((size_t)(t - 1) * M + i) * 3; /* slot 0 is the fixed start */
        for (int a = 0; a < 3; ++a) {
          gxp[a] += prm->w_coll * Ssum * dv[a];
          gxm[a] -= prm->w_coll * Ssum * dv[a];
        }
      }
    }
  }

  /* Eq. 9 self term per state (skipped whole when the caller asks for no
   * self check: IK mode without the self term, Sec. 6's IK without collision
   * checking) */
  double* gself = (double*)calloc((size_t)M * 3, sizeof(double));
  const int self_check = !(ik && !(prm->flags & CRO_SELF) && (prm->flags & CRO_NO_SELF_CHECK));
  for (int t = 1; t <= H && self_check; ++t) {
    const double* Xt = X + (size_t)t * M * 4;
    int32_t arg;
    double pen = cro_self_penetration(rb, Xt, &arg, gself);
    /* the argmax pair decides the gradient */
    if (pen > 0.0 && (prm->flags & CRO_SELF)) note_margin(&smg[t - 1], self_argmax_gap(rb, Xt));
    /* validity: every pair of S separated */
    double pair_clear = DBL_MAX;
    for (int32_t p = 0; p < rb->n_pairs; ++p) {
      int i = rb->pairs[2 * p], j = rb->pairs[2 * p + 1];
      if (Xt[4 * i + 3] <= 0.0 || Xt[4 * j + 3] <= 0.0) continue;
      double d[3] = {Xt[4 * i] - Xt[4 * j], Xt[4 * i + 1] - Xt[4 * j + 1], Xt[4 * i + 2] - Xt[4 * j + 2]};
      double clear = norm3(d) - Xt[4 * i + 3] - Xt[4 * j + 3];
      if (clear < pair_clear) pair_clear = clear;
      if (!(clear > 0.0)) free_ok = 0;
    }
    if (pair_clear < scl[t - 1]) scl[t - 1] = pair_clear;
    /* max(0, .) of Eq. 9 switches the gradient on at zero penetration */
    if (prm->flags & CRO_SELF) note_margin(&smg[t - 1], pair_clear);
    if (prm->flags & CRO_SELF) {
      ss[t - 1] = prm->w_self * pen;
      term[1] += prm->w_self * pen;
      for (int k = 0; k < M * 3; ++k) GX[(size_t)t * M * 3 + k] += prm->w_self * gself[k];
    }
  }
  free(gself);

  /* Eq. 14 goal term at the last state */
  double dp[3], dR[9];
  term[4] = cro_goal_cost(prm, ee, goal7, dp, dR);

  /* backward through the kinematics, state by state */
  double* G = (double*)calloc((size_t)H * D, sizeof(double));
  for (int t = 1; t <= H; ++t) {
    backward_state(rb, LT + (size_t)t * D * 12, X + (size_t)t * M * 4,
                   GX + (size_t)t * M * 3, t == H ? ee : NULL, dp, dR, G + (size_t)(t - 1) * D);
  }

  /* Eq. 15 joint-space goal term at the last state:
   * alpha_4 logcosh(alpha_5 |theta_g - theta_H|^2) */
  if ((prm->flags & CRO_CSPACE_GOAL) && goal_q) {
    const double* thH = theta + (size_t)(H - 1) * D;
    double r2 = 0.0;
    for (int j = 0; j < D; ++j) r2 += (thH[j] - goal_q[j]) * (thH[j] - goal_q[j]);
    term[4] += prm->w_cspace * logcosh(prm->k_cspace * r2);
    double f = prm->w_cspace * prm->k_cspace * tanh(prm->k_cspace * r2);
    for (int j = 0; j < D; ++j) G[(size_t)(H - 1) * D + j] += 2.0 * f * (thH[j] - goal_q[j]);
  }

  /* Eq. 17 position bound on theta_1..theta_H */
  for (int t = 0; t < H; ++t) {
    for (int j = 0; j < D; ++j) {
      double s;
      term[2] += prm->w_bound *
                 cro_bound_cost(theta[t * D + j], rb->q_lo[j], rb->q_hi[j], prm->eta_bound, &s);
      G[t * D + j] += prm->w_bound * s;
    }
  }

  if (!ik) {
    /* App. A.5 stencils, Eq. 16 smoothness, Eq. 17 derivative bounds */
    int NS = H + 1;
    double* vel = (double*)malloc((size_t)NS * D * sizeof(double));
    double* acc = (double*)malloc((size_t)NS * D * sizeof(double));
    double* jrk = (double*)malloc((size_t)NS * D * sizeof(double));
    double* dv = (double*)calloc((size_t)NS * D, sizeof(double));
    double* da = (double*)calloc((size_t)NS * D, sizeof(double));
    double* dj = (double*)calloc((size_t)NS * D, sizeof(double));
    cro_stencil(H, D, q_start, theta, prm->dt, vel, acc, jrk);
    for (int k = 0; k < NS * D; ++k) {
      int j = k % D;
      double s;
      term[3] += prm->w_acc * acc[k] * acc[k] + prm->w_jerk * jrk[k] * jrk[k];
      da[k] += 2.0 * prm->w_acc * acc[k];
      dj[k] += 2.0 * prm->w_jerk * jrk[k];
      if (prm->flags & CRO_VEL_COST) {
        term[3] += prm->w_vel * logcosh(prm->k_vel * vel[k]);
        dv[k] += prm->w_vel * prm->k_vel * tanh(prm->k_vel * vel[k]);
      }
      term[2] += prm->w_bound * cro_bound_cost(vel[k], -rb->v_max[j], rb->v_max[j], prm->eta_bound, &s);
      dv[k] += prm->w_bound * s;
      term[2] += prm->w_bound * cro_bound_cost(acc[k], -rb->a_max[j], rb->a_max[j], prm->eta_bound, &s);
      da[k] += prm->w_bound * s;
      term[2] += prm->w_bound * cro_bound_cost(jrk[k], -rb->j_max[j], rb->j_max[j], prm->eta_bound, &s);
      dj[k] += prm->w_bound * s;
    }
    /* transpose of the stencils onto the padded sequence, then onto theta:
     * ext index e' = t + 2 holds theta_t; H+3 and H+4 are copies of theta_H;
     * 0..2 are the fixed start state */
    const double cv[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
    const double ca[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
    const double cj[5] = {-1.0, 2.0, 0.0, -2.0, 1.0};
    double sv = 1.0 / (12.0 * prm->dt), sa = 1.0 / (12.0 * prm->dt * prm->dt),
           sj = 1.0 / (2.0 * prm->dt * prm->dt * prm->dt);
    for (int e = 2; e <= H + 2; ++e) {
      int k = e - 2;
      for (int o = -2; o <= 2; ++o) {
        int n = e + o;
        if (n <= 2) continue;                     /* start state: not a variable */
        int t = n >= H + 2 ? H : n - 2;           /* theta_t, 1-based */
        for (int j = 0; j < D; ++j) {
          G[(t - 1) * D + j] += dv[k * D + j] * cv[o + 2] * sv + da[k * D + j] * ca[o + 2] * sa +
                                dj[k * D + j] * cj[o + 2] * sj;
        }
      }
    }
    free(vel); free(acc); free(jrk); free(dv); free(da); free(dj);
  }

  double total = 0.0;
  for (int k = 0; k < CRO_N_TERMS; ++k) total += term[k];
  *cost = total;
  if (grad) memcpy(grad, G, (size_t)H * D * sizeof(double));
  if (cfree) *cfree = (uint8_t)free_ok;
  if (terms) memcpy(terms, term, sizeof(term));
  /* the trajectory's margin: every decision of every state, clearances included */
  for (int t = 0; t < H; ++t) {
    note_margin(&mg, smg[t]);
    note_margin(&mg, scl[t]);
  }
  if (margin) *margin = mg;
  if (st_terms)
    for (int t = 0; t < H; ++t) {
      st_terms[2 * t] = sw[t];
      st_terms[2 * t + 1] = ss[t];
    }
  if (st_margin) memcpy(st_margin, smg, (size_t)H * sizeof(double));
  if (st_clear) memcpy(st_clear, scl, (size_t)H * sizeof(double));
  free(sw); free(ss); free(smg); free(scl);
  free(G); free(LT); free(X); free(GX);
}

void cro_eval(const cro_robot* rb, const cro_world* w, const double* q_start, const double* goal7,
              const double* goal_q, const cro_params* prm, int32_t H, const double* theta, int32_t B,
              double* cost,
              double* grad, uint8_t* cfree, double* terms, double* margin) {
  cro_eval_states(rb, w, q_start, goal7, goal_q, prm, H, theta, B, cost, grad, cfree, terms, margin,
                  NULL, NULL, NULL);
}

void cro_eval_states(const cro_robot* rb, const cro_world* w, const double* q_start,
                     const double* goal7, const double* goal_q, const cro_params* prm, int32_t H,
                     const double* theta, int32_t B, double* cost, double* grad, uint8_t* cfree,
                     double* terms, double* margin, double* state_terms, double* state_margin,
                     double* state_clear) {
  box_t* boxes = (box_t*)malloc((size_t)(w->n > 0 ? w->n : 1) * sizeof(box_t));
  for (int k = 0; k < w->n; ++k) {
    memcpy(boxes[k].pose, w->pose + 7 * k, 7 * sizeof(double));
    memcpy(boxes[k].h, w->half_ext + 3 * k, 3 * sizeof(double));
  }
  size_t n = (size_t)H * rb->dof;
  for (int b = 0; b < B; ++b) {
    eval_one(rb, boxes, w->n, q_start, goal7, goal_q, prm, H, theta + b * n, cost + b,
             grad ? grad + b * n : NULL, cfree ? cfree + b : NULL,
             terms ? terms + (size_t)b * CRO_N_TERMS : NULL, margin ? margin + b : NULL,
             state_terms ? state_terms + (size_t)b * H * 2 : NULL,
             state_margin ? state_margin + (size_t)b * H : NULL,
             state_clear ? state_clear + (size_t)b * H : NULL);
  }
  free(boxes);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 + App. A.7 "L-BFGS Step Update" (Nocedal & Wright two-loop)        */
/* ------------------------------------------------------------------------ */

static double dotn(int32_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int32_t k = 0; k < n; ++k) s += a[k] * b[k];
  return s;
}

/* Readings: buffers start at zero with rho = 0, so unfilled pairs are inert;
 * rho = 1 / y^T s only when y^T s > 1e-8, else 0 (the pair is inert); the
 * initial Hessian H^0 = gamma I with gamma = s^T y / y^T y of the newest pair
 * with rho > 0, else 1; with no valid pair the direction is -g. */
void cro_lbfgs_direction(cro_lbfgs* st, double* d) {
  const int32_t n = st->n, m = st->m;
  if (*st->iter > 0) {
    /* shift buffers, then the newest pair at index m-1 */
    for (int32_t i = 0; i + 1 < m; ++i) {
      memcpy(st->s + (size_t)i * n, st->s + (size_t)(i + 1) * n, (size_t)n * sizeof(double));
      memcpy(st->y + (size_t)i * n, st->y + (size_t)(i + 1) * n, (size_t)n * sizeof(double));
      st->rho[i] = st->rho[i + 1];
    }
    double* s = st->s + (size_t)(m - 1) * n;
    double* y = st->y + (size_t)(m - 1) * n;
    for (int32_t k = 0; k < n; ++k) {
      s[k] = st->x[k] - st->x_prev[k];
      y[k] = st->g[k] - st->g_prev[k];
    }
    double ys = dotn(n, y, s);
    st->rho[m - 1] = ys > 1e-8 ? 1.0 / ys : 0.0;
  }
  memcpy(st->x_prev, st->x, (size_t)n * sizeof(double));
  memcpy(st->g_prev, st->g, (size_t)n * sizeof(double));
  *st->iter += 1;

  double alpha[CRO_MAX_HISTORY];
  double* q = d; /* q <- g, then the first loop from newest to oldest */
  memcpy(q, st->g, (size_t)n * sizeof(double));
  for (int32_t i = m - 1; i >= 0; --i) {
    alpha[i] = st->rho[i] * dotn(n, st->s + (size_t)i * n, q);
    for (int32_t k = 0; k < n; ++k) q[k] -= alpha[i] * st->y[(size_t)i * n + k];
  }
  double gamma = 1.0;
  for (int32_t i = m - 1; i >= 0; --i) {
    if (st->rho[i] > 0.0) {
      gamma = dotn(n, st->s + (size_t)i * n, st->y + (size_t)i * n) /
              dotn(n, st->y + (size_t)i * n, st->y + (size_t)i * n);
      break;
    }
  }
  for (int32_t k = 0; k < n; ++k) q[k] *= gamma; /* r = H^0 q */
  for (int32_t i = 0; i < m; ++i) {              /* second loop, oldest to newest */
    double beta = st->rho[i] * dotn(n, st->y + (size_t)i * n, q);
    for (int32_t k = 0; k < n; ++k) q[k] += st->s[(size_t)i * n + k] * (alpha[i] - beta);
  }
  for (int32_t k = 0; k < n; ++k) d[k] = -q[k]; /* descent direction -H g */
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 parallel noisy line search                                          */
/* ------------------------------------------------------------------------ */

void cro_ls_candidates(const cro_params* prm, int32_t n, int32_t dof, const double* q_lo,
                       const double* q_hi, const double* x, const double* d, double* cand) {
  for (int32_t l = 0; l < prm->n_alpha; ++l) {
    for (int32_t k = 0; k < n; ++k) {
      int j = k % dof;
      double v = x[k] + prm->alpha[l] * d[k];
      if (v < q_lo[j]) v = q_lo[j];
      if (v > q_hi[j]) v = q_hi[j];
      cand[(size_t)l * n + k] = v;
    }
  }
}

/* Reading of the garbled tests: Armijo c_l <= c_0 + c1 alpha_l g_0^T d;
 * weak Wolfe g_l^T d >= c2 g_0^T d; strong Wolfe |g_l^T d| <= c2 |g_0^T d|.
 * largest_true returns the largest passing index, else 0 (the 0.01 step). */
int32_t cro_ls_select(const cro_params* prm, int32_t n, double c0, const double* g0,
                      const double* d, const double* cand_cost, const double* cand_grad,
                      double* margin) {
  double gd0 = dotn(n, g0, d);
  int32_t best = 0;
  double mg = DBL_MAX;
  for (int32_t l = 0; l < prm->n_alpha; ++l) {
    double armijo = c0 + prm->armijo_c1 * prm->alpha[l] * gd0 - cand_cost[l];
    int ok = armijo >= 0.0;
    if (fabs(armijo) < mg) mg = fabs(armijo);
    if (prm->flags & CRO_WOLFE) {
      double gld = dotn(n, cand_grad + (size_t)l * n, d);
      double w;
      if (prm->flags & CRO_STRONG_WOLFE)
        w = prm->wolfe_c2 * fabs(gd0) - fabs(gld);
      else
        w = gld - prm->wolfe_c2 * gd0;
      ok = ok && (w >= 0.0);
      if (fabs(w) < mg) mg = fabs(w);
    }
    if (ok) best = l;
  }
  if (margin) *margin = mg;
  return best;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: iterations with best-iterate tracking                            */
/* ------------------------------------------------------------------------ */

void cro_solve(const cro_robot* rb, const cro_world* w, const double* q_start,
               const double* goal7, const double* goal_q, const cro_params* prm, int32_t H, int32_t B,
               const double* seeds, int32_t iters, double* best_x, double* best_c,
               uint8_t* best_cfree) {
  const int32_t D = rb->dof, n = H * D, m = prm->history, na = prm->n_alpha;
  double* x = (double*)malloc((size_t)B * n * sizeof(double));
  double* g = (double*)malloc((size_t)B * n * sizeof(double));
  double* c = (double*)malloc((size_t)B * sizeof(double));
  uint8_t* cf = (uint8_t*)malloc((size_t)B);
  double* xp = (double*)calloc((size_t)B * n, sizeof(double));
  double* gp = (double*)calloc((size_t)B * n, sizeof(double));
  double* S = (double*)calloc((size_t)B * m * n, sizeof(double));
  double* Y = (double*)calloc((size_t)B * m * n, sizeof(double));
  double* rho = (double*)calloc((size_t)B * m, sizeof(double));
  int32_t* it = (int32_t*)calloc((size_t)B, sizeof(int32_t));
  double* d = (double*)malloc((size_t)B * n * sizeof(double));
  double* cand = (double*)malloc((size_t)B * na * n * sizeof(double));
  double* cc = (double*)malloc((size_t)B * na * sizeof(double));
  double* cg = (double*)malloc((size_t)B * na * n * sizeof(double));
  uint8_t* ccf = (uint8_t*)malloc((size_t)B * na);

  memcpy(x, seeds, (size_t)B * n * sizeof(double));
  cro_eval(rb, w, q_start, goal7, goal_q, prm, H, x, B, c, g, cf, NULL, NULL);
  memcpy(best_x, x, (size_t)B * n * sizeof(double));
  memcpy(best_c, c, (size_t)B * sizeof(double));
  memcpy(best_cfree, cf, (size_t)B);

  for (int32_t iter = 0; iter < iters; ++iter) {
    for (int32_t b = 0; b < B; ++b) {
      cro_lbfgs st = {n, m, x + (size_t)b * n, g + (size_t)b * n, c + b, xp + (size_t)b * n,
                      gp + (size_t)b * n, S + (size_t)b * m * n, Y + (size_t)b * m * n,
                      rho + (size_t)b * m, it + b};
      cro_lbfgs_direction(&st, d + (size_t)b * n);
      cro_ls_candidates(prm, n, D, rb->q_lo, rb->q_hi, x + (size_t)b * n, d + (size_t)b * n,
                        cand + (size_t)b * na * n);
    }
    cro_eval(rb, w, q_start, goal7, goal_q, prm, H, cand, B * na, cc, cg, ccf, NULL, NULL);
    for (int32_t b = 0; b < B; ++b) {
      int32_t l = cro_ls_select(prm, n, c[b], g + (size_t)b * n, d + (size_t)b * n,
                                cc + (size_t)b * na, cg + (size_t)b * na * n, NULL);
      size_t src = ((size_t)b * na + l) * n;
      memcpy(x + (size_t)b * n, cand + src, (size_t)n * sizeof(double));
      memcpy(g + (size_t)b * n, cg + src, (size_t)n * sizeof(double));
      c[b] = cc[(size_t)b * na + l];
      if (c[b] < best_c[b]) { /* keep the best iterate: noisy steps may diverge */
        best_c[b] = c[b];
        memcpy(best_x + (size_t)b * n, x + (size_t)b * n, (size_t)n * sizeof(double));
        best_cfree[b] = ccf[(size_t)b * na + l];
      }
    }
  }
  free(x); free(g); free(c); free(cf); free(xp); free(gp); free(S); free(Y); free(rho); free(it);
  free(d); free(cand); free(cc); free(cg); free(ccf);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2 particle-based optimisation                                       */
/* ------------------------------------------------------------------------ */

void cro_particle_sample(int32_t n, int32_t n_p, const double* mu, const double* sigma,
                         const double* eps, double* particles) {
  for (int32_t i = 0; i < n_p; ++i)
    for (int32_t k = 0; k < n; ++k)
      particles[(size_t)i * n + k] = mu[k] + sqrt(sigma[k]) * eps[(size_t)i * n + k];
}

void cro_particle_update(int32_t n, int32_t n_p, const double* cost, const double* particles,
                         double beta, double k_mu, double k_sigma, double* mu, double* sigma,
                         double* w) {
  /* exponential utility of c = -cost / beta */
  double cmin = cost[0];
  for (int32_t i = 1; i < n_p; ++i)
    if (cost[i] < cmin) cmin = cost[i];
  double* wt = (double*)malloc((size_t)n_p * sizeof(double));
  double z = 0.0;
  for (int32_t i = 0; i < n_p; ++i) {
    wt[i] = exp(-(cost[i] - cmin) / beta);
    z += wt[i];
  }
  for (int32_t i = 0; i < n_p; ++i) wt[i] /= z;
  /* Eq. 12 and Eq. 13, both from the previous mean */
  for (int32_t k = 0; k < n; ++k) {
    double m = 0.0, v = 0.0;
    for (int32_t i = 0; i < n_p; ++i) {
      double th = particles[(size_t)i * n + k];
      m += wt[i] * th;
      v += wt[i] * (th - mu[k]) * (th - mu[k]);
    }
    sigma[k] = (1.0 - k_sigma) * sigma[k] + k_sigma * v;
    mu[k] = (1.0 - k_mu) * mu[k] + k_mu * m;
  }
  if (w) memcpy(w, wt, (size_t)n_p * sizeof(double));
  free(wt);
}

/* ------------------------------------------------------------------------ */
/* Sec. 5 Alg. "Parallel Steering"                                            */
/* ------------------------------------------------------------------------ */

int32_t cro_steer_steps(int32_t E, int32_t dof, const double* edges, double r) {
  double gmax = 0.0;
  for (int32_t e = 0; e < E; ++e)
    for (int32_t j = 0; j < dof; ++j) {
      double g = fabs(edges[((size_t)e * 2 + 1) * dof + j] - edges[((size_t)e * 2) * dof + j]);
      if (g > gmax) gmax = g;
    }
  return (int32_t)floor(gmax / r) + 1;
}

void cro_steer(const cro_robot* rb, const cro_world* w, int32_t E, const double* edges, int32_t n,
               int32_t* last, double* v_new, double* dist) {
  const int D = rb->dof;
  cro_params prm;
  cro_params_default(&prm);
  prm.flags = CRO_IK_MODE | CRO_SELF; /* single states: the discrete test only */
  const double goal7[7] = {0, 0, 0, 1, 0, 0, 0};
  double* l = (double*)malloc((size_t)D * sizeof(double));
  for (int32_t e = 0; e < E; ++e) {
    const double* a = edges + (size_t)e * 2 * D;
    const double* b = a + D;
    int32_t h = n;
    for (int32_t i = 0; i <= n; ++i) {
      for (int j = 0; j < D; ++j) l[j] = a[j] + ((double)i / n) * (b[j] - a[j]);
      double c;
      uint8_t ok;
      cro_eval(rb, w, l, goal7, NULL, &prm, 1, l, 1, &c, NULL, &ok, NULL, NULL);
      if (!ok) {
        h = i - 1;
        break;
      }
    }
    last[e] = h;
    double s = h < 0 ? 0.0 : (double)h / n, d2 = 0.0;
    for (int j = 0; j < D; ++j) {
      double v = a[j] + s * (b[j] - a[j]);
      v_new[(size_t)e * D + j] = v;
      d2 += (v - a[j]) * (v - a[j]);
    }
    dist[e] = sqrt(d2);
  }
  free(l);
}

/* ------------------------------------------------------------------------ */
/* App. "Time-step Discretization": retime                                    */
/* ------------------------------------------------------------------------ */

double cro_retime(const cro_robot* rb, int32_t H, const double* q0, const double* theta) {
  const int D = rb->dof, NS = H + 1;
  double* v = (double*)malloc((size_t)NS * D * sizeof(double));
  double* a = (double*)malloc((size_t)NS * D * sizeof(double));
  double* j = (double*)malloc((size_t)NS * D * sizeof(double));
  cro_stencil(H, D, q0, theta, 1.0, v, a, j);
  double dt = 0.0;
  for (int k = 0; k < NS * D; ++k) {
    int jj = k % D;
    double dv = fabs(v[k]) / rb->v_max[jj];
    double da = sqrt(fabs(a[k]) / rb->a_max[jj]);
    double dj = cbrt(fabs(j[k]) / rb->j_max[jj]);
    if (dv > dt) dt = dv;
    if (da > dt) dt = da;
    if (dj > dt) dt = dj;
  }
  free(v); free(a); free(j);
  return dt;
}

/* ------------------------------------------------------------------------ */
/* App. "Solver details": choosing among the seeds of a solve                 */
/* ------------------------------------------------------------------------ */

double cro_pose_error(const cro_robot* rb, const double* q, const double* goal7) {
  double* lt = (double*)malloc((size_t)rb->dof * 12 * sizeof(double));
  double* sp = (double*)malloc((size_t)(rb->n_spheres > 0 ? rb->n_spheres : 1) * 4 * sizeof(double));
  double ee[12], Rg[9];
  cro_fk(rb, q, lt, sp, ee);
  free(lt); free(sp);
  quat_to_rot(goal7 + 3, Rg);
  double e[3] = {ee[3] - goal7[0], ee[7] - goal7[1], ee[11] - goal7[2]};
  double tr = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) tr += Rg[a * 3 + b] * ee[a * 4 + b];
  return norm3(e) + (3.0 - tr) / 4.0;
}

int32_t cro_rank_seeds(const cro_robot* rb, int32_t H, int32_t B, const double* q0, const double* goal7,
                       const double* theta, const uint8_t* cfree, const double* dt, double dt_all,
                       int32_t ik, double w_pose, double w_jerk, double w_time, double w_dist, double* score) {
  const int D = rb->dof, NS = H + 1;
  double* v = (double*)malloc((size_t)NS * D * sizeof(double));
  double* a = (double*)malloc((size_t)NS * D * sizeof(double));
  double* j = (double*)malloc((size_t)NS * D * sizeof(double));
  int32_t best = -1;
  for (int b = 0; b < B; ++b) {
    const double* th = theta + (size_t)b * H * D;
    const double* last = th + (size_t)(H - 1) * D;
    double s = w_pose * cro_pose_error(rb, last, goal7);
    if (ik) {
      double d2 = 0.0;
      for (int k = 0; k < D; ++k) d2 += (last[k] - q0[k]) * (last[k] - q0[k]);
      s += w_dist * sqrt(d2);
    } else {
      const double dtb = dt ? dt[b] : dt_all;
      cro_stencil(H, D, q0, th, dtb, v, a, j);
      double jmax = 0.0;
      for (int k = 0; k < NS * D; ++k)
        if (fabs(j[k]) > jmax) jmax = fabs(j[k]);
      s += w_jerk * jmax + w_time * H * dtb;
    }
    score[b] = s;
    if (cfree[b] && !isnan(s) && (best < 0 || s < score[best])) best = b;
  }
  free(v); free(a); free(j);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Alg. "Time Discretization" (App. "Time-step Discretization")               */
/* ------------------------------------------------------------------------ */

/* Reading of "scale the weights by the new dt": the App. A.5 derivatives of
 * the same waypoints scale as 1/dt^k, so multiplying the weight on the square
 * of the k-th derivative by (dt / dt0)^(2k) keeps the term's value. */
void cro_time_scaled_params(const cro_params* prm, double dt, int32_t jerk, cro_params* out) {
  double r = dt / prm->dt;
  *out = *prm;
  out->dt = dt;
  out->w_vel = prm->w_vel * r * r;
  out->w_acc = prm->w_acc * pow(r, 4.0);
  out->w_jerk = jerk ? prm->w_jerk * pow(r, 6.0) : 0.0;
}

/* the solve's best seed: lowest-cost collision-free, else lowest-cost */
static int32_t solve_best(int32_t B, const double* cost, const uint8_t* cfree) {
  int32_t bi = 0, bf = -1;
  for (int32_t b = 0; b < B; ++b) {
    if (cost[b] < cost[bi]) bi = b;
    if (cfree[b] && (bf < 0 || cost[b] < cost[bf])) bf = b;
  }
  return bf >= 0 ? bf : bi;
}

int32_t cro_time_discretized_solve(const cro_robot* rb, const cro_world* w, const double* q_start,
                                   const double* goal7, const double* goal_q, const cro_params* prm,
                                   int32_t H, int32_t B, const double* seeds, int32_t iters1, int32_t iters2,
                                   double dt_init, double dt_min, double w_pose, double w_jerk, double w_time,
                                   double* first, double* stage, double* traj, double* cost, uint8_t* cfree,
                                   double* dt, double* score) {
  const size_t n = (size_t)H * rb->dof;
  cro_params p1, p2;
  /* 1. solve at the coarse step without the jerk term */
  cro_time_scaled_params(prm, dt_init, 0, &p1);
  double* x1 = (double*)malloc((size_t)B * n * sizeof(double));
  double* c1 = (double*)malloc((size_t)B * sizeof(double));
  uint8_t* f1 = (uint8_t*)malloc((size_t)B);
  cro_solve(rb, w, q_start, goal7, goal_q, &p1, H, B, seeds, iters1, x1, c1, f1);
  /* 2. retime the best seed; scale the weights to that step, jerk on */
  int32_t b1 = solve_best(B, c1, f1);
  double dt_opt = cro_retime(rb, H, q_start, x1 + (size_t)b1 * n);
  if (dt_opt < dt_min) dt_opt = dt_min;
  cro_time_scaled_params(prm, dt_opt, 1, &p2);
  if (first) memcpy(first, x1 + (size_t)b1 * n, n * sizeof(double));
  if (stage) {
    stage[0] = p1.dt; stage[1] = p1.w_vel; stage[2] = p1.w_acc; stage[3] = p1.w_jerk;
    stage[4] = p2.dt; stage[5] = p2.w_vel; stage[6] = p2.w_acc; stage[7] = p2.w_jerk;
  }
  /* 3. solve again from every seed of the first solve */
  cro_solve(rb, w, q_start, goal7, goal_q, &p2, H, B, x1, iters2, traj, cost, cfree);
  /* 4. retime every seed, score it at its own step, choose */
  for (int32_t b = 0; b < B; ++b) dt[b] = cro_retime(rb, H, q_start, traj + (size_t)b * n);
  int32_t chosen = cro_rank_seeds(rb, H, B, q_start, goal7, traj, cfree, dt, 0.0, 0, w_pose, w_jerk, w_time,
                                  0.0, score);
  if (chosen < 0) chosen = solve_best(B, cost, cfree);
  free(x1); free(c1); free(f1);
  return chosen;
}
