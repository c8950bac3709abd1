/*
 * inhand_oracle.c -- plain, slow FP64 CPU oracle of the in-hand tracking hot
 * path (arXiv 2002.12160, "In-Hand Object Pose Tracking via Contact Feedback
 * and GPU-Accelerated Robotic Simulation").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path calls this file: it is
 * used by tests/, by the smoke check and by the CPU-baseline leg of the
 * benchmark. It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, step by step, in the order of the paper's Algorithm 1:
 *   f(s_t, u_t, theta)   the dynamics step (Sec. III-A), here a kinematic hand,
 *                        sphere-cluster object, brute-force contact enumeration,
 *                        a fixed-iteration Jacobi projected impulse solve with
 *                        Coulomb friction, and symplectic Euler integration;
 *   o_t^(i)              the contact-sensor force c_t^(l) of every pad (Sec. III-A);
 *   C_i, i*              windowed mean cost and argmin (Eqs. 1-2, Sec. III-C);
 *   opt(...)             the periodic resample + perturbation (Sec. III-D,
 *                        population-based variant with elite weighting);
 *   p_0^(i) ~ N(p_0, Sigma_p), theta ~ theta_0   initial sampling (Sec. III-D).
 * The paper does not fix the solver, the bias, the inertia of a sphere cluster,
 * the sensor threshold, the elite weights or the random stream; this file takes
 * the readings listed in the design notes and nothing else.
 *
 * Every function works on one environment at a time with plain loops; there is
 * no blocking, fusion or reordering beyond what the equations state.
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, brute force, library routines or published vectors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* records passed from Python (ctypes mirrors live in oracle/__init__.py)    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t n_shapes;
    const int32_t *shape_first;   /* [n_shapes] */
    const int32_t *shape_count;   /* [n_shapes] */
    const double *spheres;        /* [total][4] body-frame centre, radius */
    double palm_half[3];
    int32_t n_fingers;
    const double *finger_root;    /* [F][4] x, y, z, yaw */
    double link_len, link_rad;
    int32_t n_pads;
    const int32_t *pad_link;
    const double *pad_s0, *pad_s1;
} orc_scene;

typedef struct {
    double frame_dt;
    int32_t substeps, iters;
    double margin, beta, slop, vmax;
    double gravity[3];
    double tau, w_force, w_contact;
    int32_t c_max;
    double escape_radius;
} orc_config;

typedef struct {
    double elite_frac;
    double floor_std[8];
    double m_lo, m_hi, mu_lo, mu_hi;
} orc_opt;

enum { ORC_NONFINITE = 1, ORC_ESCAPED = 2, ORC_OVERFLOW = 4 };
#define ORC_DIVERGED (ORC_NONFINITE | ORC_ESCAPED | ORC_OVERFLOW)

/* ------------------------------------------------------------------------- */
/* small FP64 linear algebra                                                  */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } vec3;
typedef struct { double w, x, y, z; } quat;
typedef struct { double m[3][3]; } mat3;

static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vscale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double vnorm(vec3 a) { return sqrt(vdot(a, a)); }
static vec3 vcross(vec3 a, vec3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

static quat qmul(quat a, quat b) {
    quat r;
    r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
    r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
    r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
    r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
    return r;
}
static quat qconj(quat a) { quat r = {a.w, -a.x, -a.y, -a.z}; return r; }
static quat qnormalize(quat a) {
    double n = sqrt(a.w * a.w + a.x * a.x + a.y * a.y + a.z * a.z);
    quat r = {a.w / n, a.x / n, a.y / n, a.z / n};
    return r;
}
/* rotation matrix of a unit quaternion */
static mat3 qmat(quat q) {
    mat3 R;
    double w = q.w, x = q.x, y = q.y, z = q.z;
    R.m[0][0] = 1 - 2 * (y * y + z * z); R.m[0][1] = 2 * (x * y - w * z); R.m[0][2] = 2 * (x * z + w * y);
    R.m[1][0] = 2 * (x * y + w * z); R.m[1][1] = 1 - 2 * (x * x + z * z); R.m[1][2] = 2 * (y * z - w * x);
    R.m[2][0] = 2 * (x * z - w * y); R.m[2][1] = 2 * (y * z + w * x); R.m[2][2] = 1 - 2 * (x * x + y * y);
    return R;
}
static vec3 mvmul(mat3 A, vec3 v) {
    return v3(A.m[0][0] * v.x + A.m[0][1] * v.y + A.m[0][2] * v.z,
              A.m[1][0] * v.x + A.m[1][1] * v.y + A.m[1][2] * v.z,
              A.m[2][0] * v.x + A.m[2][1] * v.y + A.m[2][2] * v.z);
}
static vec3 mtvmul(mat3 A, vec3 v) { /* A^T v */
    return v3(A.m[0][0] * v.x + A.m[1][0] * v.y + A.m[2][0] * v.z,
              A.m[0][1] * v.x + A.m[1][1] * v.y + A.m[2][1] * v.z,
              A.m[0][2] * v.x + A.m[1][2] * v.y + A.m[2][2] * v.z);
}
static mat3 mmul(mat3 A, mat3 B) {
    mat3 C;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A.m[i][k] * B.m[k][j];
            C.m[i][j] = s;
        }
    return C;
}
static mat3 mtrans(mat3 A) {
    mat3 T;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T.m[i][j] = A.m[j][i];
    return T;
}
/* skew matrix [r]x with [r]x v = r x v */
static mat3 skew(vec3 r) {
    mat3 S = {{{0, -r.z, r.y}, {r.z, 0, -r.x}, {-r.y, r.x, 0}}};
    return S;
}
/* inverse by the adjugate: A^-1 = adj(A) / det(A) */
static mat3 minv(mat3 A) {
    double (*a)[3] = A.m;
    mat3 C;
    C.m[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    C.m[0][1] = a[0][2] * a[2][1] - a[0][1] * a[2][2];
    C.m[0][2] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
    C.m[1][0] = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    C.m[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
    C.m[1][2] = a[0][2] * a[1][0] - a[0][0] * a[1][2];
    C.m[2][0] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    C.m[2][1] = a[0][1] * a[2][0] - a[0][0] * a[2][1];
    C.m[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
    double det = a[0][0] * C.m[0][0] + a[0][1] * C.m[1][0] + a[0][2] * C.m[2][0];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) C.m[i][j] /= det;
    return C;
}

/* so(3) exponential as a unit quaternion: rotation by |w| about w/|w| */
static quat quat_exp(vec3 w) {
    double th = vnorm(w);
    quat r;
    if (th < 1e-300) { r.w = 1; r.x = r.y = r.z = 0; return r; }
    double s = sin(0.5 * th) / th;
    r.w = cos(0.5 * th); r.x = w.x * s; r.y = w.y * s; r.z = w.z * s;
    return r;
}
/* so(3) logarithm of a unit quaternion (shortest rotation vector) */
static vec3 quat_log(quat q) {
    if (q.w < 0) { q.w = -q.w; q.x = -q.x; q.y = -q.y; q.z = -q.z; }
    double s = sqrt(q.x * q.x + q.y * q.y + q.z * q.z);
    if (s < 1e-300) return v3(0, 0, 0);
    double th = 2.0 * atan2(s, q.w);
    return v3(q.x * th / s, q.y * th / s, q.z * th / s);
}

/* ------------------------------------------------------------------------- */
/* 4x4 homogeneous transforms for the finger kinematics                       */
/* ------------------------------------------------------------------------- */
typedef struct { double m[4][4]; } mat4;

static mat4 m4_identity(void) {
    mat4 T; memset(&T, 0, sizeof T);
    for (int i = 0; i < 4; i++) T.m[i][i] = 1;
    return T;
}
static mat4 m4_mul(mat4 A, mat4 B) {
    mat4 C;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double s = 0;
            for (int k = 0; k < 4; k++) s += A.m[i][k] * B.m[k][j];
            C.m[i][j] = s;
        }
    return C;
}
static mat4 m4_trans(double x, double y, double z) {
    mat4 T = m4_identity();
    T.m[0][3] = x; T.m[1][3] = y; T.m[2][3] = z;
    return T;
}
static mat4 m4_rotz(double a) {
    mat4 T = m4_identity();
    T.m[0][0] = cos(a); T.m[0][1] = -sin(a);
    T.m[1][0] = sin(a); T.m[1][1] = cos(a);
    return T;
}
static mat4 m4_roty(double a) {
    mat4 T = m4_identity();
    T.m[0][0] = cos(a); T.m[0][2] = sin(a);
    T.m[2][0] = -sin(a); T.m[2][2] = cos(a);
    return T;
}
/* rotation matrix -> unit quaternion (w >= 0), by the largest-diagonal branch */
static quat mat_to_quat(const double R[3][3]) {
    quat q;
    double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        double s = 2.0 * sqrt(1.0 + tr);
        q.w = 0.25 * s;
        q.x = (R[2][1] - R[1][2]) / s; q.y = (R[0][2] - R[2][0]) / s; q.z = (R[1][0] - R[0][1]) / s;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double s = 2.0 * sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
        q.w = (R[2][1] - R[1][2]) / s; q.x = 0.25 * s;
        q.y = (R[0][1] + R[1][0]) / s; q.z = (R[0][2] + R[2][0]) / s;
    } else if (R[1][1] > R[2][2]) {
        double s = 2.0 * sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]);
        q.w = (R[0][2] - R[2][0]) / s; q.x = (R[0][1] + R[1][0]) / s;
        q.y = 0.25 * s; q.z = (R[1][2] + R[2][1]) / s;
    } else {
        double s = 2.0 * sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]);
        q.w = (R[1][0] - R[0][1]) / s; q.x = (R[0][2] + R[2][0]) / s;
        q.y = (R[1][2] + R[2][1]) / s; q.z = 0.25 * s;
    }
    if (q.w < 0) { q.w = -q.w; q.x = -q.x; q.y = -q.y; q.z = -q.z; }
    return qnormalize(q);
}

/*
 * Kinematic hand (the robot state of Sec. III-A driven by desired joint
 * positions u_t). Link 0 is the palm box at the origin. Finger f has links
 * 1 + 4f + j, j = 0..3, each a capsule of length L along its frame's +x:
 *   T_0 = Trans(root) Rz(yaw + q0) Ry(-pi/2)      (upright knuckle link)
 *   T_j = T_{j-1} Trans(L, 0, 0) Ry(-q_j), j=1..3 (flexion curls inward)
 * Output: per link, position xyz and quaternion wxyz (7 doubles).
 */
int orc_fk(const orc_scene *sc, const double *q, double *link_pose) {
    double *o = link_pose;
    o[0] = o[1] = o[2] = 0; o[3] = 1; o[4] = o[5] = o[6] = 0;
    for (int f = 0; f < sc->n_fingers; f++) {
        const double *rt = sc->finger_root + 4 * f;
        const double *qf = q + 4 * f;
        mat4 T = m4_mul(m4_mul(m4_trans(rt[0], rt[1], rt[2]), m4_rotz(rt[3] + qf[0])),
                        m4_roty(-M_PI / 2));
        for (int j = 0; j < 4; j++) {
            if (j > 0) T = m4_mul(m4_mul(T, m4_trans(sc->link_len, 0, 0)), m4_roty(-qf[j]));
            double R[3][3];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) R[a][b] = T.m[a][b];
            quat qq = mat_to_quat(R);
            double *p = link_pose + 7 * (1 + 4 * f + j);
            p[0] = T.m[0][3]; p[1] = T.m[1][3]; p[2] = T.m[2][3];
            p[3] = qq.w; p[4] = qq.x; p[5] = qq.y; p[6] = qq.z;
        }
    }
    return 0;
}

typedef struct { vec3 p; quat q; mat3 R; } pose_t;

static pose_t pose_from7(const double *p7) {
    pose_t P;
    P.p = v3(p7[0], p7[1], p7[2]);
    P.q.w = p7[3]; P.q.x = p7[4]; P.q.y = p7[5]; P.q.z = p7[6];
    P.R = qmat(P.q);
    return P;
}

/* ------------------------------------------------------------------------- */
/* narrowphase: one sphere (world centre c, radius rs) against one link       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double d;        /* signed gap: surface distance, negative = penetration */
    vec3 n;          /* unit normal pointing from the link to the object */
    double t;        /* axial parameter along the capsule, 0 for the palm */
    double face_gap; /* palm, centre inside: gap between the two shallowest faces */
} np_hit;

/* sphere vs capsule: closest point on the segment a..b, clamp t to [0, 1] */
static np_hit sphere_capsule(vec3 c, double rs, vec3 a, vec3 b, double rc, quat link_q) {
    np_hit h;
    vec3 ab = vsub(b, a);
    double t = vdot(vsub(c, a), ab) / vdot(ab, ab);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    vec3 closest = vadd(a, vscale(ab, t));
    vec3 diff = vsub(c, closest);
    double dist = vnorm(diff);
    h.t = t;
    h.face_gap = INFINITY;
    if (dist < 1e-9) {
        /* centre on the axis: use the link-local +z direction */
        h.n = mvmul(qmat(link_q), v3(0, 0, 1));
    } else {
        h.n = vscale(diff, 1.0 / dist);
    }
    h.d = dist - rs - rc;
    return h;
}

/* sphere vs oriented box: clamp the centre into the box in box coordinates */
static np_hit sphere_box(vec3 c, double rs, pose_t box, const double half[3]) {
    np_hit h;
    vec3 cl = mtvmul(box.R, vsub(c, box.p));
    double cc[3] = {cl.x, cl.y, cl.z}, q[3];
    int inside = 1;
    for (int i = 0; i < 3; i++) {
        q[i] = cc[i];
        if (q[i] > half[i]) { q[i] = half[i]; inside = 0; }
        if (q[i] < -half[i]) { q[i] = -half[i]; inside = 0; }
    }
    h.t = 0;
    h.face_gap = INFINITY;
    if (!inside) {
        vec3 diff = v3(cc[0] - q[0], cc[1] - q[1], cc[2] - q[2]);
        double dist = vnorm(diff);
        h.n = mvmul(box.R, vscale(diff, 1.0 / dist));
        h.d = dist - rs;
    } else {
        /* shallowest of the six faces; ties go to the lowest axis, + side first */
        double best = INFINITY, second = INFINITY;
        int axis = 0; double sgn = 1;
        for (int i = 0; i < 3; i++) {
            double dp = half[i] - cc[i], dm = half[i] + cc[i];
            if (dp < best) { second = best; best = dp; axis = i; sgn = 1; }
            else if (dp < second) second = dp;
            if (dm < best) { second = best; best = dm; axis = i; sgn = -1; }
            else if (dm < second) second = dm;
        }
        double nl[3] = {0, 0, 0};
        nl[axis] = sgn;
        h.n = mvmul(box.R, v3(nl[0], nl[1], nl[2]));
        h.d = -best - rs;
        h.face_gap = second - best;
    }
    return h;
}

/* link l against a world sphere; link poses are (pos, quat) 7-vectors */
static np_hit link_hit(const orc_scene *sc, int l, const double *link_pose, vec3 c, double rs) {
    pose_t P = pose_from7(link_pose + 7 * l);
    if (l == 0) return sphere_box(c, rs, P, sc->palm_half);
    vec3 a = P.p;
    vec3 b = vadd(P.p, mvmul(P.R, v3(sc->link_len, 0, 0)));
    return sphere_capsule(c, rs, a, b, sc->link_rad, P.q);
}

/* sensor pad of a contact on link l at axial parameter t (first match wins) */
static int pad_of(const orc_scene *sc, int l, double t) {
    for (int k = 0; k < sc->n_pads; k++) {
        if (sc->pad_link[k] != l) continue;
        if (l == 0) return k;
        if (t >= sc->pad_s0[k] && (t < sc->pad_s1[k] || sc->pad_s1[k] >= 1.0)) return k;
    }
    return -1;
}

static double pad_boundary_gap(const orc_scene *sc, int l, double t) {
    double g = INFINITY;
    if (l == 0) return g;
    for (int k = 0; k < sc->n_pads; k++) {
        if (sc->pad_link[k] != l) continue;
        if (sc->pad_s0[k] > 0) g = fmin(g, fabs(t - sc->pad_s0[k]));
        if (sc->pad_s1[k] < 1) g = fmin(g, fabs(t - sc->pad_s1[k]));
    }
    return g * sc->link_len;
}

/*
 * Brute-force contact list of one object (shape s at pose7) against every
 * link: every (sphere, link) pair is tested, no culling. A pair is a contact
 * when d < margin. Row layout of `out` (12 doubles): sphere, link, pad, d,
 * n xyz, p xyz (the object sphere's point closest to the link), t.
 * Returns the number of contacts (rows beyond max_out are counted, not written).
 */
int orc_contacts(const orc_scene *sc, const orc_config *cfg, int shape, const double *pose7,
                 const double *link_pose, int max_out, double *out) {
    pose_t X = pose_from7(pose7);
    int first = sc->shape_first[shape], cnt = sc->shape_count[shape];
    int n_links = 1 + 4 * sc->n_fingers, nc = 0;
    /* body offsets are taken relative to the sphere-centre centroid */
    vec3 cen = v3(0, 0, 0);
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        cen = vadd(cen, v3(s[0], s[1], s[2]));
    }
    cen = vscale(cen, 1.0 / cnt);
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        vec3 c = vadd(X.p, mvmul(X.R, vsub(v3(s[0], s[1], s[2]), cen)));
        for (int l = 0; l < n_links; l++) {
            np_hit h = link_hit(sc, l, link_pose, c, s[3]);
            if (!(h.d < cfg->margin)) continue;
            if (nc < max_out) {
                double *o = out + 12 * nc;
                vec3 p = vsub(c, vscale(h.n, s[3]));
                o[0] = j; o[1] = l; o[2] = pad_of(sc, l, h.t); o[3] = h.d;
                o[4] = h.n.x; o[5] = h.n.y; o[6] = h.n.z;
                o[7] = p.x; o[8] = p.y; o[9] = p.z; o[10] = h.t; o[11] = 0;
            }
            nc++;
        }
    }
    return nc;
}

/*
 * Unit inertia of a sphere cluster about its centroid (inertia per unit
 * mass): every sphere carries 1/S of the mass as a solid ball,
 *   J = (1/S) sum_s [ (2/5) r_s^2 I + |c_s|^2 I - c_s c_s^T ],
 * with c_s measured from the centroid of the sphere centres.
 */
int orc_unit_inertia(const orc_scene *sc, int shape, double *J9) {
    int first = sc->shape_first[shape], cnt = sc->shape_count[shape];
    vec3 cen = v3(0, 0, 0);
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        cen = vadd(cen, v3(s[0], s[1], s[2]));
    }
    cen = vscale(cen, 1.0 / cnt);
    double J[3][3] = {{0}};
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        vec3 c = vsub(v3(s[0], s[1], s[2]), cen);
        double cv[3] = {c.x, c.y, c.z};
        double ball = 0.4 * s[3] * s[3] + vdot(c, c);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) J[a][b] += ((a == b) ? ball : 0.0) - cv[a] * cv[b];
    }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) J9[3 * a + b] = J[a][b] / cnt;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* the dynamics step f(s_t, u_t, theta) for one environment over one frame    */
/* ------------------------------------------------------------------------- */
typedef struct {
    vec3 r, n, vl;   /* lever arm, normal, link point velocity */
    double inv_kn;   /* 1 / (n^T K n): normal step */
    double inv_kt;   /* 1 / ((tr K - n^T K n) / 2): tangential step */
    double b;        /* velocity bias along n */
    int pad;
    int id;          /* pair id: link << 8 | sphere */
    vec3 lam;        /* accumulated impulse on the object */
    vec3 lam_next;   /* this iteration's update (Jacobi: applied after all k) */
} contact_t;

/* Warm start: the final impulses of the environment's previous substep, by
 * pair id (n entries). Each contact of the next substep starts from its
 * pair's impulse if the pair was a contact then, else from zero. */
typedef struct {
    int32_t *n;       /* entries */
    int32_t *id;      /* [cap] pair ids */
    double *lam;      /* [cap][3] impulses */
    int cap;
} lam_cache;

static vec3 cache_lookup(const lam_cache *c, int id) {
    for (int k = 0; k < *c->n; k++)
        if (c->id[k] == id) return v3(c->lam[3 * k], c->lam[3 * k + 1], c->lam[3 * k + 2]);
    return v3(0, 0, 0);
}

/*
 * One contact's projected update from the current impulse lam and relative
 * velocity u: a scalar effective-mass step along the normal, clamped at zero,
 * and a scalar step in the tangent plane, clamped radially to the Coulomb disk
 * of radius mu * lambda_n. Scalar (per direction) steps make the fixed point
 * the discrete Coulomb solution: u_n + b = 0 where lambda_n > 0, u_t = 0 where
 * the contact sticks, and lambda_t opposite to u_t where it slides.
 */
static vec3 contact_update(vec3 lam, vec3 u, vec3 n, double b, double inv_kn, double inv_kt,
                           double mu) {
    double un = vdot(u, n);
    vec3 ut = vsub(u, vscale(n, un));
    double ln = vdot(lam, n) - (un + b) * inv_kn;
    if (ln < 0) ln = 0;
    vec3 lt = vsub(vsub(lam, vscale(n, vdot(lam, n))), vscale(ut, inv_kt));
    double tn = vnorm(lt);
    if (tn > mu * ln) lt = (tn > 0) ? vscale(lt, mu * ln / tn) : v3(0, 0, 0);
    return vadd(vscale(n, ln), lt);
}

/* velocity bias: speculative approach when separated, slop, clamped recovery */
static double contact_bias(const orc_config *cfg, double d, double h) {
    if (d > 0) return d / h;
    double b = cfg->beta * fmin(d + cfg->slop, 0.0) / h;
    return fmax(b, -cfg->vmax);
}

/*
 * Velocity of a point p on a link over a substep of length h: the point is
 * carried rigidly from the link's pose A (substep start, 7 doubles: position,
 * quaternion w x y z) to its pose B (substep end), and the velocity is the
 * displacement over h:  v = (p_B - p) / h,  p_B = B.p + B.R A.R^T (p - A.p).
 */
void orc_link_point_velocity(const double *A7, const double *B7, const double *p3, double h, double *out3) {
    pose_t A = pose_from7(A7), B = pose_from7(B7);
    vec3 p = v3(p3[0], p3[1], p3[2]);
    vec3 pl = mtvmul(A.R, vsub(p, A.p));         /* in link coords */
    vec3 p1 = vadd(B.p, mvmul(B.R, pl));         /* carried to the end */
    vec3 v = vscale(vsub(p1, p), 1.0 / h);
    out3[0] = v.x; out3[1] = v.y; out3[2] = v.z;
}

/* per-environment diagnostics written by orc_step (doubles per env) */
#define ORC_DIAG 6  /* contacts (sum over substeps), pair tests, min|d-margin|,
                       min pad-boundary gap (m), min face gap (m), iterations */

static void step_env(const orc_scene *sc, const orc_config *cfg, const double *lp_all,
                     int ns, double *pose7, double *vel6, const double *theta,
                     int shape, int iters, int32_t *status, double *forces, double *diag,
                     contact_t *ct, int ct_cap, const lam_cache *cache) {
    const int n_links = 1 + 4 * sc->n_fingers;
    const int P = sc->n_pads;
    const double h = cfg->frame_dt / ns;
    const double m = theta[0], mu = theta[1];
    const vec3 g = v3(cfg->gravity[0], cfg->gravity[1], cfg->gravity[2]);
    for (int k = 0; k < 3 * P; k++) forces[k] = 0;
    diag[0] = 0; diag[1] = 0; diag[2] = INFINITY; diag[3] = INFINITY; diag[4] = INFINITY;
    diag[5] = 0;
    if (*status & ORC_DIVERGED) return;   /* replaced at the next optimizer update */

    int first = sc->shape_first[shape], cnt = sc->shape_count[shape];
    vec3 cen = v3(0, 0, 0);
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        cen = vadd(cen, v3(s[0], s[1], s[2]));
    }
    cen = vscale(cen, 1.0 / cnt);
    double J9[9];
    orc_unit_inertia(sc, shape, J9);
    mat3 J;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) J.m[a][b] = J9[3 * a + b];
    mat3 Jinv = minv(J);

    vec3 x = v3(pose7[0], pose7[1], pose7[2]);
    quat q = {pose7[3], pose7[4], pose7[5], pose7[6]};
    vec3 v = v3(vel6[0], vel6[1], vel6[2]);
    vec3 w = v3(vel6[3], vel6[4], vel6[5]);

    for (int s = 0; s < ns; s++) {
        const double *lp0 = lp_all + (size_t)s * n_links * 7;       /* substep start */
        const double *lp1 = lp_all + (size_t)(s + 1) * n_links * 7; /* substep end */
        /* gravity prediction; no gyroscopic term */
        vec3 v_pred = vadd(v, vscale(g, h));
        vec3 w_pred = w;
        mat3 R = qmat(q);
        /* world inverse inertia W = R J^-1 R^T / m */
        mat3 W = mmul(mmul(R, Jinv), mtrans(R));
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) W.m[a][b] /= m;

        /* brute-force contact generation over every (sphere, link) pair */
        int nc = 0;
        for (int j = 0; j < cnt; j++) {
            const double *sp = sc->spheres + 4 * (first + j);
            vec3 c = vadd(x, mvmul(R, vsub(v3(sp[0], sp[1], sp[2]), cen)));
            for (int l = 0; l < n_links; l++) {
                np_hit hh = link_hit(sc, l, lp0, c, sp[3]);
                diag[1] += 1;
                double gap = fabs(hh.d - cfg->margin);
                if (gap < diag[2]) diag[2] = gap;
                if (!(hh.d < cfg->margin)) continue;
                if (hh.face_gap < diag[4]) diag[4] = hh.face_gap;
                double pg = pad_boundary_gap(sc, l, hh.t);
                if (pg < diag[3]) diag[3] = pg;
                if (nc < ct_cap) {
                    contact_t *k = &ct[nc];
                    vec3 p = vsub(c, vscale(hh.n, sp[3]));
                    k->r = vsub(p, x);
                    k->n = hh.n;
                    k->pad = pad_of(sc, l, hh.t);
                    /* K = (1/m) I - [r]x W [r]x, the contact-point inverse mass */
                    mat3 S = skew(k->r);
                    mat3 K = mmul(mmul(S, W), S);
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            K.m[a][b] = ((a == b) ? 1.0 / m : 0.0) - K.m[a][b];
                    double kn = vdot(k->n, mvmul(K, k->n));
                    double kt = 0.5 * (K.m[0][0] + K.m[1][1] + K.m[2][2] - kn);
                    k->inv_kn = 1.0 / kn;
                    k->inv_kt = 1.0 / kt;
                    k->b = contact_bias(cfg, hh.d, h);
                    /* link point velocity from the link's rigid displacement */
                    if (l == 0) {
                        k->vl = v3(0, 0, 0);
                    } else {
                        double pp[3] = {p.x, p.y, p.z}, vv[3];
                        orc_link_point_velocity(lp0 + 7 * l, lp1 + 7 * l, pp, h, vv);
                        k->vl = v3(vv[0], vv[1], vv[2]);
                    }
                    k->id = (l << 8) | j;
                    k->lam = cache ? cache_lookup(cache, k->id) : v3(0, 0, 0);
                }
                nc++;
            }
        }
        diag[0] += nc;
        if (nc > cfg->c_max) {   /* more contacts than the per-env capacity */
            *status |= ORC_OVERFLOW;
            nc = 0;
        }

        /* Jacobi projected impulse iterations with 1/n_c relaxation */
        for (int it = 0; it < iters && nc > 0; it++) {
            vec3 F = v3(0, 0, 0), Tq = v3(0, 0, 0);
            for (int k = 0; k < nc; k++) {
                F = vadd(F, ct[k].lam);
                Tq = vadd(Tq, vcross(ct[k].r, ct[k].lam));
            }
            vec3 vi = vadd(v_pred, vscale(F, 1.0 / m));
            vec3 wi = vadd(w_pred, mvmul(W, Tq));
            for (int k = 0; k < nc; k++) {
                contact_t *c = &ct[k];
                vec3 u = vsub(vadd(vi, vcross(wi, c->r)), c->vl);
                vec3 lproj = contact_update(c->lam, u, c->n, c->b, c->inv_kn, c->inv_kt, mu);
                c->lam_next = vadd(c->lam, vscale(vsub(lproj, c->lam), 1.0 / nc));
            }
            for (int k = 0; k < nc; k++) ct[k].lam = ct[k].lam_next;
            diag[5] += 1;
        }
        vec3 F = v3(0, 0, 0), Tq = v3(0, 0, 0);
        for (int k = 0; k < nc; k++) {
            F = vadd(F, ct[k].lam);
            Tq = vadd(Tq, vcross(ct[k].r, ct[k].lam));
        }
        v = vadd(v_pred, vscale(F, 1.0 / m));
        w = vadd(w_pred, mvmul(W, Tq));

        /* symplectic Euler: position with the new velocity, exact rotation */
        x = vadd(x, vscale(v, h));
        q = qnormalize(qmul(quat_exp(vscale(w, h)), q));

        /* sensor pads: force on the pad by the object is -lambda / h */
        for (int k = 0; k < nc; k++) {
            if (ct[k].pad < 0) continue;
            double *fp = forces + 3 * ct[k].pad;
            fp[0] -= ct[k].lam.x / h; fp[1] -= ct[k].lam.y / h; fp[2] -= ct[k].lam.z / h;
        }
        /* the warm-start cache: this substep's contacts and final impulses */
        if (cache) {
            int nk = nc < cache->cap ? nc : cache->cap;
            for (int k = 0; k < nk; k++) {
                cache->id[k] = ct[k].id;
                cache->lam[3 * k] = ct[k].lam.x; cache->lam[3 * k + 1] = ct[k].lam.y; cache->lam[3 * k + 2] = ct[k].lam.z;
            }
            *cache->n = nk;
        }
    }
    for (int k = 0; k < 3 * P; k++) forces[k] /= ns;

    pose7[0] = x.x; pose7[1] = x.y; pose7[2] = x.z;
    pose7[3] = q.w; pose7[4] = q.x; pose7[5] = q.y; pose7[6] = q.z;
    vel6[0] = v.x; vel6[1] = v.y; vel6[2] = v.z; vel6[3] = w.x; vel6[4] = w.y; vel6[5] = w.z;
    int finite = 1;
    for (int k = 0; k < 7; k++) finite &= isfinite(pose7[k]);
    for (int k = 0; k < 6; k++) finite &= isfinite(vel6[k]);
    if (!finite) *status |= ORC_NONFINITE;
    else if (vnorm(x) > cfg->escape_radius) *status |= ORC_ESCAPED;
}

/*
 * Step N environments over frames [frame0, frame0 + n_frames). The commanded
 * joint angles are given at the frame boundaries (q_traj[(frames+1)][D]);
 * within a frame the hand moves linearly in joint space, so substep k of ns
 * uses q = q_f + (k/ns)(q_{f+1} - q_f).
 * pose [N][7] (xyz, wxyz), vel [N][6] (linear, angular, world frame),
 * theta [N][2] (mass, friction), shape [N], iters [N] or NULL (cfg->iters),
 * status [N] (sticky bits), forces [N][P][3] of the last frame stepped,
 * diag [N][ORC_DIAG] of the last frame stepped. With cache_n non-NULL the
 * solver is warm-started: cache_n [N], cache_id [N][cache_cap] and
 * cache_lam [N][cache_cap][3] carry each environment's last substep's
 * contacts (pair id = link << 8 | sphere) and final impulses, read at the
 * next substep and rewritten after it.
 */
int orc_step(const orc_scene *sc, const orc_config *cfg, int N, const double *q_traj,
             int frame0, int n_frames, double *pose, double *vel, const double *theta,
             const int32_t *shape, const int32_t *iters, int32_t *status, double *forces,
             double *diag, int32_t *cache_n, int32_t *cache_id, double *cache_lam, int cache_cap) {
    const int D = 4 * sc->n_fingers, n_links = 1 + 4 * sc->n_fingers, ns = cfg->substeps;
    const int P = sc->n_pads;
    double *lp = (double *)malloc(sizeof(double) * 7 * n_links * (ns + 1));
    double *qk = (double *)malloc(sizeof(double) * (D > 0 ? D : 1));
    int cap = 1;
    for (int s = 0; s < sc->n_shapes; s++) cap = cap > sc->shape_count[s] ? cap : sc->shape_count[s];
    cap = cap * n_links + 1;       /* every (sphere, link) pair */
    contact_t *ct = (contact_t *)malloc(sizeof(contact_t) * cap);
    for (int f = frame0; f < frame0 + n_frames; f++) {
        for (int k = 0; k <= ns; k++) {
            for (int j = 0; j < D; j++) {
                double q0 = q_traj[(size_t)f * D + j], q1 = q_traj[(size_t)(f + 1) * D + j];
                qk[j] = q0 + ((double)k / ns) * (q1 - q0);
            }
            orc_fk(sc, qk, lp + (size_t)k * n_links * 7);
        }
        for (int i = 0; i < N; i++) {
            int it = iters ? iters[i] : cfg->iters;
            lam_cache c = {cache_n + i, cache_id + (size_t)i * cache_cap, cache_lam + (size_t)i * 3 * cache_cap,
                           cache_cap};
            step_env(sc, cfg, lp, ns, pose + 7 * (size_t)i, vel + 6 * (size_t)i,
                     theta + 2 * (size_t)i, shape ? shape[i] : 0, it, status + i,
                     forces + (size_t)i * 3 * P, diag + (size_t)i * ORC_DIAG, ct, cap,
                     cache_n ? &c : NULL);
        }
    }
    free(lp); free(qk); free(ct);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* cost (Sec. III-C, force and contact-state terms) and argmin (Eqs. 1-2)     */
/* ------------------------------------------------------------------------- */

/* per-frame cost of one environment against the observation */
static double frame_cost(const orc_config *cfg, int P, const double *c_sim, const double *c_obs) {
    double cost = 0;
    for (int l = 0; l < P; l++) {
        const double *a = c_sim + 3 * l, *b = c_obs + 3 * l;
        double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
        cost += cfg->w_force * (dx * dx + dy * dy + dz * dz);
        /* a sensor is in contact when its force magnitude exceeds tau,
           i.e. when the squared magnitude exceeds tau^2 (Sec. III-C) */
        double na2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        double nb2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        double tau2 = cfg->tau * cfg->tau;
        int in_a = na2 > tau2, in_b = nb2 > tau2;
        if (in_a != in_b) cost += cfg->w_contact;   /* w (1 - alpha) */
    }
    return cost;
}

/*
 * Adds this frame's cost to c_sum (running sum since the window start) and
 * returns i* = argmin_i c_sum[i] / n_window (NaN counts as +inf, ties go to
 * the lowest index). Diverged environments cost +inf. cost_out [N] (may be
 * NULL) receives this frame's per-environment cost.
 */
int orc_cost(const orc_config *cfg, int N, int P, const double *forces, const double *obs,
             const int32_t *status, double *c_sum, int n_window, double *c_mean, double *cost_out) {
    int best = 0;
    double best_c = INFINITY;
    for (int i = 0; i < N; i++) {
        double c = (status[i] & ORC_DIVERGED) ? INFINITY : frame_cost(cfg, P, forces + (size_t)3 * P * i, obs);
        if (cost_out) cost_out[i] = c;
        c_sum[i] += c;
        double cm = c_sum[i] / n_window;
        if (c_mean) c_mean[i] = cm;
        if (isnan(cm)) cm = INFINITY;
        if (cm < best_c || (i == 0)) { best_c = cm; best = i; }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* counter-based random numbers: Philox4x32-10 (Salmon et al., SC'11)         */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* the four 32-bit words of block (stream, index, env, block) under seed */
static void rng_block(uint64_t seed, uint32_t stream, uint32_t index, uint32_t env, uint32_t blk,
                      uint32_t out[4]) {
    uint32_t ctr[4] = {stream, index, env, blk};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}
/* uniform in (0, 1) from 53 bits of two words */
static double u01(uint32_t hi, uint32_t lo) {
    uint64_t bits = ((uint64_t)hi << 21) | (lo >> 11);
    return ((double)bits + 0.5) * (1.0 / 9007199254740992.0);
}
/* two standard normals by the Box-Muller transform */
static void box_muller(const uint32_t w[4], double *z0, double *z1) {
    double a = u01(w[0], w[1]), b = u01(w[2], w[3]);
    double rad = sqrt(-2.0 * log(a));
    *z0 = rad * cos(2.0 * M_PI * b);
    *z1 = rad * sin(2.0 * M_PI * b);
}

/* n standard normals of (stream, index, env), two per Philox block */
int orc_normals(uint64_t seed, uint32_t stream, uint32_t index, uint32_t env, int n, double *out) {
    for (int k = 0; k < n; k += 2) {
        uint32_t w[4];
        double a, b;
        rng_block(seed, stream, index, env, (uint32_t)(k / 2), w);
        box_muller(w, &a, &b);
        out[k] = a;
        if (k + 1 < n) out[k + 1] = b;
    }
    return 0;
}

/* uniforms in (0,1): two per block, block `blk` of (stream, index, env) */
int orc_uniforms(uint64_t seed, uint32_t stream, uint32_t index, uint32_t env, uint32_t blk, double *out2) {
    uint32_t w[4];
    rng_block(seed, stream, index, env, blk, w);
    out2[0] = u01(w[0], w[1]);
    out2[1] = u01(w[2], w[3]);
    return 0;
}

/*
 * Initial sampling (Sec. III-D; Algorithm 1, initialisation):
 *   x0^(i) = x0 + sigma_p n_{0..2},  R0^(i) = exp([sigma_r n_{3..5}]x) R0,
 *   m ~ U[m_lo, m_hi], mu ~ U[mu_lo, mu_hi]
 * with n from stream 0, index 0, env i, blocks 0..2 and the two uniforms from
 * block 3.
 */
int orc_sample_initial(int N, const double *nominal7, double sigma_p, double sigma_r,
                       double m_lo, double m_hi, double mu_lo, double mu_hi, uint64_t seed,
                       double *pose, double *theta) {
    quat q0 = {nominal7[3], nominal7[4], nominal7[5], nominal7[6]};
    for (int i = 0; i < N; i++) {
        double n[6], u[2];
        orc_normals(seed, 0, 0, (uint32_t)i, 6, n);
        orc_uniforms(seed, 0, 0, (uint32_t)i, 3, u);
        double *p = pose + 7 * (size_t)i;
        p[0] = nominal7[0] + sigma_p * n[0];
        p[1] = nominal7[1] + sigma_p * n[1];
        p[2] = nominal7[2] + sigma_p * n[2];
        quat q = qnormalize(qmul(quat_exp(v3(sigma_r * n[3], sigma_r * n[4], sigma_r * n[5])), q0));
        p[3] = q.w; p[4] = q.x; p[5] = q.y; p[6] = q.z;
        theta[2 * i] = m_lo + (m_hi - m_lo) * u[0];
        theta[2 * i + 1] = mu_lo + (mu_hi - mu_lo) * u[1];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* optimizer update (Sec. III-D, PBO with elite-weighted Gaussian exploration) */
/* ------------------------------------------------------------------------- */

/* 8x8 Cholesky A = L L^T (row-major, lower), returns -1 if not positive definite */
int orc_cholesky8(const double *A, double *L) {
    for (int k = 0; k < 64; k++) L[k] = 0;
    for (int i = 0; i < 8; i++)
        for (int j = 0; j <= i; j++) {
            double s = A[8 * i + j];
            for (int k = 0; k < j; k++) s -= L[8 * i + k] * L[8 * j + k];
            if (i == j) {
                if (!(s > 0)) return -1;
                L[8 * i + i] = sqrt(s);
            } else {
                L[8 * i + j] = s / L[8 * j + j];
            }
        }
    return 0;
}

static int cmp_idx_cost(const double *C, int a, int b) {
    double ca = isnan(C[a]) ? INFINITY : C[a], cb = isnan(C[b]) ? INFINITY : C[b];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a < b) ? -1 : (a > b);
}

/*
 * One optimizer update over N environments with window-mean costs C [N].
 *  1. order by (C, index), NaN = +inf; the first k = max(1, floor(frac N))
 *     are the elites, the first of them is i*;
 *  2. elite weights w_j = exp(-(C_j - C_min) / s), s = standard deviation of
 *     the finite elite costs (uniform when s < 1e-12), normalised;
 *  3. z_j = [x_j, log(R_j R_{i*}^T), m_j, mu_j]; weighted mean and covariance
 *     Sigma_w = sum w_j (z_j - zbar)(z_j - zbar)^T; L = chol(Sigma_w + Sigma_floor);
 *  4. the non-elites, in index order r = 0..N-k-1, take parents by systematic
 *     resampling over the elites in index order: position (u + r) / (N - k),
 *     u from stream 2, block 0 of (update_index, env 0);
 *  5. each non-elite copies its parent's pose, velocity, parameters and status
 *     and adds delta = L eps, eps ~ N(0, I_8) from stream 1 (update_index,
 *     env): x += delta_0..2, R <- exp([delta_3..5]x) R, m += delta_6,
 *     mu += delta_7, then m and mu are clamped; elites are kept unchanged.
 * Outputs: parent [N] (self for elites), stats (8 means, 64 covariance, 64 L,
 * k, i*, s) in `stats` (139 doubles, may be NULL). Returns i* or -1 if the
 * Cholesky failed.
 */
int orc_optimizer(const orc_opt *op, int N, const double *C, double *pose, double *vel,
                  double *theta, int32_t *status, uint64_t seed, uint32_t update_index,
                  int32_t *parent, double *stats) {
    int *order = (int *)malloc(sizeof(int) * N);
    for (int i = 0; i < N; i++) order[i] = i;
    /* insertion sort by (C, index): plain and obviously a total order */
    for (int i = 1; i < N; i++) {
        int key = order[i], j = i - 1;
        while (j >= 0 && cmp_idx_cost(C, order[j], key) > 0) { order[j + 1] = order[j]; j--; }
        order[j + 1] = key;
    }
    int k = (int)floor(op->elite_frac * N);
    if (k < 1) k = 1;
    int istar = order[0];
    char *is_elite = (char *)calloc(N, 1);
    for (int j = 0; j < k; j++) is_elite[order[j]] = 1;

    /* elite list in index order with its weights */
    int *el = (int *)malloc(sizeof(int) * k);
    double *w = (double *)malloc(sizeof(double) * k);
    int ne = 0;
    for (int i = 0; i < N; i++) if (is_elite[i]) el[ne++] = i;
    double cmin = isnan(C[istar]) ? INFINITY : C[istar];
    double mean = 0; int nfin = 0;
    for (int j = 0; j < k; j++) if (isfinite(C[el[j]])) { mean += C[el[j]]; nfin++; }
    double sd = 0;
    if (nfin > 0) {
        mean /= nfin;
        for (int j = 0; j < k; j++) if (isfinite(C[el[j]])) sd += (C[el[j]] - mean) * (C[el[j]] - mean);
        sd = sqrt(sd / nfin);
    }
    double wsum = 0;
    for (int j = 0; j < k; j++) {
        double c = C[el[j]];
        if (nfin == 0) w[j] = 1.0;
        else if (!isfinite(c)) w[j] = 0.0;
        else if (!(sd >= 1e-12)) w[j] = 1.0;
        else w[j] = exp(-(c - cmin) / sd);
        wsum += w[j];
    }
    for (int j = 0; j < k; j++) w[j] /= wsum;

    /* weighted mean and covariance of z over the elites (zero weights skipped) */
    quat qref = {pose[7 * istar + 3], pose[7 * istar + 4], pose[7 * istar + 5], pose[7 * istar + 6]};
    double zbar[8] = {0}, cov[64] = {0}, z[8];
    for (int j = 0; j < k; j++) {
        if (w[j] == 0) continue;
        const double *p = pose + 7 * (size_t)el[j];
        quat qj = {p[3], p[4], p[5], p[6]};
        vec3 lr = quat_log(qmul(qj, qconj(qref)));
        z[0] = p[0]; z[1] = p[1]; z[2] = p[2]; z[3] = lr.x; z[4] = lr.y; z[5] = lr.z;
        z[6] = theta[2 * el[j]]; z[7] = theta[2 * el[j] + 1];
        for (int a = 0; a < 8; a++) zbar[a] += w[j] * z[a];
    }
    for (int j = 0; j < k; j++) {
        if (w[j] == 0) continue;
        const double *p = pose + 7 * (size_t)el[j];
        quat qj = {p[3], p[4], p[5], p[6]};
        vec3 lr = quat_log(qmul(qj, qconj(qref)));
        z[0] = p[0]; z[1] = p[1]; z[2] = p[2]; z[3] = lr.x; z[4] = lr.y; z[5] = lr.z;
        z[6] = theta[2 * el[j]]; z[7] = theta[2 * el[j] + 1];
        for (int a = 0; a < 8; a++)
            for (int b = 0; b < 8; b++) cov[8 * a + b] += w[j] * (z[a] - zbar[a]) * (z[b] - zbar[b]);
    }
    double A[64], L[64];
    for (int a = 0; a < 64; a++) A[a] = cov[a];
    for (int a = 0; a < 8; a++) A[9 * a] += op->floor_std[a] * op->floor_std[a];
    int chol_ok = orc_cholesky8(A, L);

    /* systematic resampling of the non-elites over the elite weights */
    double cdf_u[2];
    orc_uniforms(seed, 2, update_index, 0, 0, cdf_u);
    double u = cdf_u[0];
    int M = N - k, r = 0;
    for (int i = 0; i < N; i++) {
        if (is_elite[i]) { if (parent) parent[i] = i; continue; }
        double pos = (u + r) / M;
        double cum = 0;
        int par = el[k - 1];
        for (int j = 0; j < k; j++) {
            cum += w[j];
            if (pos < cum) { par = el[j]; break; }
        }
        r++;
        if (parent) parent[i] = par;
    }
    /* copy-and-perturb; elites are never written, so parents stay intact */
    for (int i = 0; i < N && chol_ok == 0; i++) {
        if (is_elite[i]) continue;
        int par = parent ? parent[i] : i;
        double eps[8], d[8];
        orc_normals(seed, 1, update_index, (uint32_t)i, 8, eps);
        for (int a = 0; a < 8; a++) {
            d[a] = 0;
            for (int b = 0; b <= a; b++) d[a] += L[8 * a + b] * eps[b];
        }
        double *pi = pose + 7 * (size_t)i;
        const double *pp = pose + 7 * (size_t)par;
        pi[0] = pp[0] + d[0]; pi[1] = pp[1] + d[1]; pi[2] = pp[2] + d[2];
        quat qp = {pp[3], pp[4], pp[5], pp[6]};
        quat qn = qnormalize(qmul(quat_exp(v3(d[3], d[4], d[5])), qp));
        pi[3] = qn.w; pi[4] = qn.x; pi[5] = qn.y; pi[6] = qn.z;
        for (int a = 0; a < 6; a++) vel[6 * (size_t)i + a] = vel[6 * (size_t)par + a];
        double mm = theta[2 * par] + d[6], mu = theta[2 * par + 1] + d[7];
        theta[2 * i] = fmin(fmax(mm, op->m_lo), op->m_hi);
        theta[2 * i + 1] = fmin(fmax(mu, op->mu_lo), op->mu_hi);
        status[i] = status[par];
    }
    if (stats) {
        for (int a = 0; a < 8; a++) stats[a] = zbar[a];
        for (int a = 0; a < 64; a++) stats[8 + a] = cov[a];
        for (int a = 0; a < 64; a++) stats[72 + a] = L[a];
        stats[136] = k; stats[137] = istar; stats[138] = sd;
    }
    free(order); free(is_elite); free(el); free(w);
    return chol_ok == 0 ? istar : -1;
}

/* ------------------------------------------------------------------------- */
/* WRS and REPS updates (Sec. III-D): a PMF over all simulations, K draws     */
/* with replacement, exploration of every simulation                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t kind;             /* 1 = WRS, 2 = REPS */
    double lambda;            /* WRS temperature */
    double epsilon;           /* REPS bound on KL(P || uniform) */
    double sigma_pose[6];     /* exploration: x y z (m), rotation (rad) x3 */
    double sigma_theta[2];    /* exploration: m (kg), mu */
    int32_t explore_velocity; /* 0: perturb the pose; 1: perturb the velocity instead */
    double sigma_vel[6];      /* velocity kick: linear (m/s) x3, angular (rad/s) x3 */
    double m_lo, m_hi, mu_lo, mu_hi;
} orc_soft_opt;

/* REPS sums over the finite costs at temperature eta: with D_i = C_min - C_i,
 * e_i = exp(D_i / eta): S0 = sum e_i, S1 = sum e_i D_i, S2 = sum e_i D_i^2 */
static void reps_sums(int N, const double *C, double cmin, double eta, double *S0, double *S1, double *S2) {
    double a = 0, b = 0, c = 0;
    for (int i = 0; i < N; i++) {
        if (!isfinite(C[i])) continue;
        double d = cmin - C[i], e = exp(d / eta);
        a += e; b += e * d; c += e * d * d;
    }
    *S0 = a; *S1 = b; *S2 = c;
}

/* d/d eta of the REPS dual g(eta) = eta eps + eta log((1/K) sum exp(R_i/eta)),
 * R_i = C_max + C_min - C_i (so R_i - max R = D_i):
 *   g'(eta) = eps + log(S0/K) - S1 / (eta S0) */
static double reps_dg(double eps, double K, double S0, double S1, double eta) {
    return eps + log(S0 / K) - S1 / (eta * S0);
}

/*
 * eta* = argmin_{eta > 0} g(eta) for the finite costs C (K = their count).
 * g is convex; g' rises from eps + log(n_min/K) (eta -> 0, n_min = number of
 * costs equal to C_min) to eps (eta -> inf). Returns +inf when every finite
 * cost is equal (any eta gives the uniform PMF) and 0 when
 * eps >= log(K/n_min) (the PMF concentrates on the minima). Otherwise the root
 * of g' by Newton steps in t = log(eta) (dg'/dt = Var_w(D)/eta^2), kept inside
 * a bracket that every step shrinks, bisecting when Newton leaves it.
 */
double orc_reps_eta(int N, const double *C, double eps, int *iters_out) {
    double cmin = INFINITY, cmax = -INFINITY;
    int K = 0;
    for (int i = 0; i < N; i++)
        if (isfinite(C[i])) { K++; if (C[i] < cmin) cmin = C[i]; if (C[i] > cmax) cmax = C[i]; }
    if (iters_out) *iters_out = 0;
    if (K == 0 || !(cmax > cmin)) return INFINITY;
    int nmin = 0;
    for (int i = 0; i < N; i++) if (isfinite(C[i]) && C[i] == cmin) nmin++;
    if (eps >= log((double)K / nmin)) return 0.0;
    const double range = cmax - cmin;
    double tlo = log(range) - 50.0, thi = log(range) + 50.0;   /* g'(e^tlo) < 0 < g'(e^thi) */
    double S0, S1, S2;
    for (int k = 0; k < 200; k++) {   /* widen the bracket until it holds the root */
        reps_sums(N, C, cmin, exp(tlo), &S0, &S1, &S2);
        if (reps_dg(eps, K, S0, S1, exp(tlo)) < 0) break;
        tlo -= 50.0;
    }
    double t = 0.5 * (tlo + thi);
    int it = 0;
    for (; it < 200; it++) {
        const double eta = exp(t);
        reps_sums(N, C, cmin, eta, &S0, &S1, &S2);
        const double g1 = reps_dg(eps, K, S0, S1, eta);
        if (g1 < 0) tlo = t; else thi = t;
        const double mean = S1 / S0, var = S2 / S0 - mean * mean;
        const double slope = var / (eta * eta);   /* dg'/dt */
        double tn = (slope > 0) ? t - g1 / slope : 0.5 * (tlo + thi);
        if (!(tn > tlo && tn < thi)) tn = 0.5 * (tlo + thi);
        if (fabs(tn - t) <= 1e-13 * (1.0 + fabs(t)) || thi - tlo <= 1e-13 * (1.0 + fabs(t))) { t = tn; it++; break; }
        t = tn;
    }
    if (iters_out) *iters_out = it;
    return exp(t);
}

/*
 * One WRS or REPS update over N environments with window-mean costs C [N]:
 *  1. the PMF over the finite-cost simulations (diverged ones get 0):
 *     WRS  P(i) ~ exp(-lambda (C_i - C_min));
 *     REPS P(i) ~ exp(R_i / eta*) = exp(-(C_i - C_min) / eta*), eta* from
 *          orc_reps_eta (uniform when eta* = +inf, on the minima when eta* = 0);
 *     every cost non-finite: uniform over all;
 *  2. K = N draws with replacement: environment i takes the parent at the
 *     inverse CDF (index order) of u_i, u_i from stream 3 (update_index, i);
 *  3. each environment copies its parent's pose, velocity, parameters and
 *     status (from the state before the update) and explores with eps ~ N(0, I_8)
 *     from stream 1 (update_index, i): m += s_m eps_6, mu += s_mu eps_7
 *     (clamped); pose: x += s_p,0..2 eps_0..2, R <- exp([s_r,0..2 eps_3..5]x) R,
 *     or with explore_velocity v += s_v,0..2 eps_0..2, w += s_v,3..5 eps_3..5.
 * i* = lowest (C, index). Outputs: parent [N]; stats (may be NULL): eta*,
 * sum of weights, KL(P || uniform over the finite ones), number finite,
 * C_min, C_max, Newton iterations. Returns i*.
 */
int orc_softmax_update(const orc_soft_opt *op, int N, const double *C, double *pose, double *vel,
                       double *theta, int32_t *status, uint64_t seed, uint32_t update_index,
                       int32_t *parent, double *stats) {
    int istar = 0;
    for (int i = 1; i < N; i++) if (cmp_idx_cost(C, i, istar) < 0) istar = i;
    double cmin = INFINITY, cmax = -INFINITY;
    int K = 0;
    for (int i = 0; i < N; i++)
        if (isfinite(C[i])) { K++; if (C[i] < cmin) cmin = C[i]; if (C[i] > cmax) cmax = C[i]; }
    double *w = (double *)malloc(sizeof(double) * N);
    double eta = NAN;
    int iters = 0;
    if (K == 0) {
        for (int i = 0; i < N; i++) w[i] = 1.0;
    } else if (op->kind == 2) {
        eta = orc_reps_eta(N, C, op->epsilon, &iters);
        for (int i = 0; i < N; i++) {
            if (!isfinite(C[i])) w[i] = 0.0;
            else if (isinf(eta)) w[i] = 1.0;
            else if (eta == 0.0) w[i] = (C[i] == cmin) ? 1.0 : 0.0;
            else w[i] = exp((cmin - C[i]) / eta);
        }
    } else {
        for (int i = 0; i < N; i++) w[i] = isfinite(C[i]) ? exp(-op->lambda * (C[i] - cmin)) : 0.0;
    }
    double W = 0;
    for (int i = 0; i < N; i++) W += w[i];
    double kl = 0;
    for (int i = 0; i < N; i++)
        if (w[i] > 0) kl += (w[i] / W) * log((w[i] / W) * (K > 0 ? K : N));
    /* the state before the update: every environment is replaced */
    double *p0 = (double *)malloc(sizeof(double) * 7 * N);
    double *v0 = (double *)malloc(sizeof(double) * 6 * N);
    double *t0 = (double *)malloc(sizeof(double) * 2 * N);
    int32_t *s0 = (int32_t *)malloc(sizeof(int32_t) * N);
    memcpy(p0, pose, sizeof(double) * 7 * N);
    memcpy(v0, vel, sizeof(double) * 6 * N);
    memcpy(t0, theta, sizeof(double) * 2 * N);
    memcpy(s0, status, sizeof(int32_t) * N);
    for (int i = 0; i < N; i++) {
        double u[2];
        orc_uniforms(seed, 3, update_index, (uint32_t)i, 0, u);
        const double pos = u[0] * W;
        double cum = 0;
        int par = N - 1;
        while (par > 0 && w[par] == 0) par--;   /* the last positive weight, if pos reaches W */
        for (int j = 0; j < N; j++) {
            cum += w[j];
            if (pos < cum) { par = j; break; }
        }
        if (parent) parent[i] = par;
        double eps[8];
        orc_normals(seed, 1, update_index, (uint32_t)i, 8, eps);
        const double *pp = p0 + 7 * (size_t)par;
        double *pi = pose + 7 * (size_t)i;
        double *vi = vel + 6 * (size_t)i;
        for (int a = 0; a < 6; a++) vi[a] = v0[6 * (size_t)par + a];
        if (op->explore_velocity) {
            for (int a = 0; a < 7; a++) pi[a] = pp[a];
            for (int a = 0; a < 6; a++) vi[a] += op->sigma_vel[a] * eps[a];
        } else {
            pi[0] = pp[0] + op->sigma_pose[0] * eps[0];
            pi[1] = pp[1] + op->sigma_pose[1] * eps[1];
            pi[2] = pp[2] + op->sigma_pose[2] * eps[2];
            quat qp = {pp[3], pp[4], pp[5], pp[6]};
            quat qn = qnormalize(qmul(quat_exp(v3(op->sigma_pose[3] * eps[3], op->sigma_pose[4] * eps[4],
                                                  op->sigma_pose[5] * eps[5])), qp));
            pi[3] = qn.w; pi[4] = qn.x; pi[5] = qn.y; pi[6] = qn.z;
        }
        theta[2 * i] = fmin(fmax(t0[2 * par] + op->sigma_theta[0] * eps[6], op->m_lo), op->m_hi);
        theta[2 * i + 1] = fmin(fmax(t0[2 * par + 1] + op->sigma_theta[1] * eps[7], op->mu_lo), op->mu_hi);
        status[i] = s0[par];
    }
    if (stats) {
        stats[0] = eta; stats[1] = W; stats[2] = kl; stats[3] = K; stats[4] = cmin; stats[5] = cmax;
        stats[6] = iters;
    }
    free(w); free(p0); free(v0); free(t0); free(s0);
    return istar;
}

/* ------------------------------------------------------------------------- */
/* ADD (Sec. IV): mean distance of the object's points at two poses           */
/* ------------------------------------------------------------------------- */
double orc_add(const orc_scene *sc, int shape, const double *pose_a7, const double *pose_b7) {
    pose_t A = pose_from7(pose_a7), B = pose_from7(pose_b7);
    int first = sc->shape_first[shape], cnt = sc->shape_count[shape];
    vec3 cen = v3(0, 0, 0);
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        cen = vadd(cen, v3(s[0], s[1], s[2]));
    }
    cen = vscale(cen, 1.0 / cnt);
    double sum = 0;
    for (int j = 0; j < cnt; j++) {
        const double *s = sc->spheres + 4 * (first + j);
        vec3 c = vsub(v3(s[0], s[1], s[2]), cen);
        vec3 pa = vadd(A.p, mvmul(A.R, c)), pb = vadd(B.p, mvmul(B.R, c));
        sum += vnorm(vsub(pa, pb));
    }
    return sum / cnt;
}

/* exported so tests can pin the so(3) maps against an independent library */
int orc_quat_exp(const double *w3, double *q4) {
    quat q = quat_exp(v3(w3[0], w3[1], w3[2]));
    q4[0] = q.w; q4[1] = q.x; q4[2] = q.y; q4[3] = q.z;
    return 0;
}
int orc_quat_log(const double *q4, double *w3) {
    quat q = {q4[0], q4[1], q4[2], q4[3]};
    vec3 w = quat_log(q);
    w3[0] = w.x; w3[1] = w.y; w3[2] = w.z;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* PD-driven articulated hand (the robot's joints as dynamic bodies)          */
/* ------------------------------------------------------------------------- */
/*
 * The hand's state is part of s_t (Sec. III-A: joint angles of articulated
 * bodies) and the action u_t is the desired joint position, tracked by a
 * joint-angle PD controller (Sec. IV). Every finger joint is a revolute joint
 * with a scalar inertia I (the joint-space mass matrix is taken diagonal; the
 * hand's own gravity and velocity-product terms are left to the controller).
 * The PD force is integrated implicitly over a substep of length h,
 *     I (qd' - qd) = h [kp (u - q - h qd') - kd qd'] + (contact impulses),
 * so without contact qd* = (I qd + h kp (u - q)) / M with M = I + h kd + h^2 kp,
 * and an impulse lambda on the object at the link point p acts as -lambda on
 * the link: joint a of the link's finger, proximal to (or at) the link, gets
 * -(J_a . lambda) / M with J_a = z_a x (p - o_a) (axis z_a through o_a). The
 * link point then moves with v_l = sum_a J_a qd_a, and the contact's
 * effective mass gains sum_a J_a J_a^T / M. After the solve, q += h qd.
 *
 * Observation of each pad l at the end of a frame (o_t, Sec. III-A):
 *   q_t; the pad's position P (link origin + the middle of its axial interval
 *   along the capsule; the palm's top centre) and rotation R (the link's);
 *   c (as in the kinematic step); slip: over the frame's substeps, the
 *   normal-impulse-weighted mean of the object's tangential velocity
 *   relative to the link at the pad's contacts, v_t, of the mean normal n,
 *   and of the relative spin (w - w_link) . n. The pad slips translationally
 *   when |v_t| > v_slip, with direction d = the unit 2-vector of v_t in the
 *   pad's contact plane (e1 = the link's axis projected into the plane,
 *   e2 = n x e1); it slips rotationally when |spin| > w_slip, r = [spin > 0].
 */
typedef struct {
    double kp, kd, armature;  /* N m/rad, N m s/rad, kg m^2 */
    double v_slip, w_slip;    /* m/s, rad/s */
} orc_pd;

typedef struct { vec3 z, o; } joint_t;

/* axis and origin of every finger joint from the link poses of orc_fk:
   joint 0 turns about the world z at the finger root (Rz(yaw + q0)), joint
   j >= 1 by -q_j about the y axis of link j's frame, through link j's origin */
static void joint_frames(const orc_scene *sc, const double *lp, joint_t *J) {
    for (int f = 0; f < sc->n_fingers; f++) {
        const double *rt = sc->finger_root + 4 * f;
        J[4 * f].z = v3(0, 0, 1);
        J[4 * f].o = v3(rt[0], rt[1], rt[2]);
        for (int j = 1; j < 4; j++) {
            pose_t P = pose_from7(lp + 7 * (1 + 4 * f + j));
            J[4 * f + j].z = v3(-P.R.m[0][1], -P.R.m[1][1], -P.R.m[2][1]);
            J[4 * f + j].o = P.p;
        }
    }
}

typedef struct {
    contact_t c;
    vec3 p;          /* world contact point (on the object's sphere) */
    int j0, nj;      /* joints j0 .. j0 + nj - 1 move the contact's link */
    vec3 J[4];       /* J_a = z_a x (p - o_a) */
} pd_contact_t;

/* link point velocity of a contact for joint velocities qd */
static vec3 pd_link_vel(const pd_contact_t *k, const double *qd) {
    vec3 v = v3(0, 0, 0);
    for (int a = 0; a < k->nj; a++) v = vadd(v, vscale(k->J[a], qd[k->j0 + a]));
    return v;
}

/* joint velocities for the current impulses: qd* - M^-1 sum_k J_k^T lambda_k */
static void pd_joint_vel(const pd_contact_t *ct, int nc, const double *qd_star, double M, int D, double *qd) {
    for (int a = 0; a < D; a++) qd[a] = qd_star[a];
    for (int k = 0; k < nc; k++)
        for (int a = 0; a < ct[k].nj; a++) qd[ct[k].j0 + a] -= vdot(ct[k].J[a], ct[k].c.lam) / M;
}

/* pad pose from link poses: position and quaternion (7 doubles) */
static void pad_pose_of(const orc_scene *sc, int pad, const double *lp, double *out7) {
    int l = sc->pad_link[pad];
    pose_t P = pose_from7(lp + 7 * l);
    vec3 c;
    if (l == 0) {
        c = vadd(P.p, mvmul(P.R, v3(0, 0, sc->palm_half[2])));
    } else {
        double s1 = sc->pad_s1[pad] < 1.0 ? sc->pad_s1[pad] : 1.0;
        double s0 = sc->pad_s0[pad] > 0.0 ? sc->pad_s0[pad] : 0.0;
        c = vadd(P.p, mvmul(P.R, v3(0.5 * (s0 + s1) * sc->link_len, 0, 0)));
    }
    out7[0] = c.x; out7[1] = c.y; out7[2] = c.z;
    out7[3] = P.q.w; out7[4] = P.q.x; out7[5] = P.q.y; out7[6] = P.q.z;
}

/* one environment over one frame; u_all [ns+1][D] are the desired joint
   positions at the substep boundaries */
static void step_env_pd(const orc_scene *sc, const orc_config *cfg, const orc_pd *pd, const double *u_all,
                        int ns, double *pose7, double *vel6, const double *theta, int shape, int iters,
                        int32_t *status, double *qj, double *qdj, double *forces, double *pad_pose,
                        double *slip_d, int32_t *slip_flags, double *slip_mag, double *diag, pd_contact_t *ct,
                        int ct_cap, double *last_ct, int32_t *last_n, int last_cap) {
    const int n_links = 1 + 4 * sc->n_fingers, D = 4 * sc->n_fingers;
    const int P = sc->n_pads;
    const double h = cfg->frame_dt / ns;
    const double m = theta[0], mu = theta[1];
    const vec3 g = v3(cfg->gravity[0], cfg->gravity[1], cfg->gravity[2]);
    const double M = pd->armature + h * pd->kd + h * h * pd->kp;
    double *lp = (double *)malloc(sizeof(double) * 7 * n_links);
    joint_t *JF = (joint_t *)malloc(sizeof(joint_t) * (D > 0 ? D : 1));
    double *qd_star = (double *)malloc(sizeof(double) * (D > 0 ? D : 1));
    double *qd = (double *)malloc(sizeof(double) * (D > 0 ? D : 1));
    double *acc = (double *)calloc((size_t)P * 8, sizeof(double));   /* per pad: w, vt(3), n(3), spin */
    for (int k = 0; k < 3 * P; k++) forces[k] = 0;
    for (int k = 0; k < 2 * P; k++) slip_d[k] = 0;
    for (int k = 0; k < P; k++) slip_flags[k] = 0;
    for (int k = 0; k < 2 * P; k++) slip_mag[k] = 0;
    diag[0] = 0; diag[1] = 0; diag[2] = INFINITY; diag[3] = INFINITY; diag[4] = INFINITY; diag[5] = 0;
    if (last_n) *last_n = 0;

    if (!(*status & ORC_DIVERGED)) {
        int first = sc->shape_first[shape], cnt = sc->shape_count[shape];
        vec3 cen = v3(0, 0, 0);
        for (int j = 0; j < cnt; j++) {
            const double *s = sc->spheres + 4 * (first + j);
            cen = vadd(cen, v3(s[0], s[1], s[2]));
        }
        cen = vscale(cen, 1.0 / cnt);
        double J9[9];
        orc_unit_inertia(sc, shape, J9);
        mat3 Jb;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Jb.m[a][b] = J9[3 * a + b];
        mat3 Jinv = minv(Jb);
        vec3 x = v3(pose7[0], pose7[1], pose7[2]);
        quat q = {pose7[3], pose7[4], pose7[5], pose7[6]};
        vec3 v = v3(vel6[0], vel6[1], vel6[2]);
        vec3 w = v3(vel6[3], vel6[4], vel6[5]);

        for (int s = 0; s < ns; s++) {
            const double *u1 = u_all + (size_t)(s + 1) * D;
            orc_fk(sc, qj, lp);              /* the hand at the substep start */
            joint_frames(sc, lp, JF);
            for (int a = 0; a < D; a++)
                qd_star[a] = (pd->armature * qdj[a] + h * pd->kp * (u1[a] - qj[a])) / M;
            vec3 v_pred = vadd(v, vscale(g, h));
            vec3 w_pred = w;
            mat3 R = qmat(q);
            mat3 W = mmul(mmul(R, Jinv), mtrans(R));
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) W.m[a][b] /= m;

            int nc = 0;
            for (int j = 0; j < cnt; j++) {
                const double *sp = sc->spheres + 4 * (first + j);
                vec3 c = vadd(x, mvmul(R, vsub(v3(sp[0], sp[1], sp[2]), cen)));
                for (int l = 0; l < n_links; l++) {
                    np_hit hh = link_hit(sc, l, lp, c, sp[3]);
                    diag[1] += 1;
                    double gap = fabs(hh.d - cfg->margin);
                    if (gap < diag[2]) diag[2] = gap;
                    if (!(hh.d < cfg->margin)) continue;
                    if (hh.face_gap < diag[4]) diag[4] = hh.face_gap;
                    double pg = pad_boundary_gap(sc, l, hh.t);
                    if (pg < diag[3]) diag[3] = pg;
                    if (nc < ct_cap) {
                        pd_contact_t *k = &ct[nc];
                        vec3 p = vsub(c, vscale(hh.n, sp[3]));
                        k->p = p;
                        k->c.r = vsub(p, x);
                        k->c.n = hh.n;
                        k->c.pad = pad_of(sc, l, hh.t);
                        k->c.id = (l << 8) | j;
                        k->c.lam = v3(0, 0, 0);
                        k->c.b = contact_bias(cfg, hh.d, h);
                        k->j0 = 0; k->nj = 0;
                        if (l > 0) {
                            k->j0 = 4 * ((l - 1) / 4);
                            k->nj = (l - 1) % 4 + 1;
                            for (int a = 0; a < k->nj; a++)
                                k->J[a] = vcross(JF[k->j0 + a].z, vsub(p, JF[k->j0 + a].o));
                        }
                        /* K = (1/m) I - [r]x W [r]x + sum_a J_a J_a^T / M */
                        mat3 S = skew(k->c.r);
                        mat3 K = mmul(mmul(S, W), S);
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++) K.m[a][b] = ((a == b) ? 1.0 / m : 0.0) - K.m[a][b];
                        for (int a = 0; a < k->nj; a++) {
                            double Ja[3] = {k->J[a].x, k->J[a].y, k->J[a].z};
                            for (int r1 = 0; r1 < 3; r1++)
                                for (int r2 = 0; r2 < 3; r2++) K.m[r1][r2] += Ja[r1] * Ja[r2] / M;
                        }
                        double kn = vdot(k->c.n, mvmul(K, k->c.n));
                        double kt = 0.5 * (K.m[0][0] + K.m[1][1] + K.m[2][2] - kn);
                        k->c.inv_kn = 1.0 / kn;
                        k->c.inv_kt = 1.0 / kt;
                    }
                    nc++;
                }
            }
            diag[0] += nc;
            if (nc > cfg->c_max) {
                *status |= ORC_OVERFLOW;
                nc = 0;
            }

            /* Jacobi iterations over object and joint velocities together */
            for (int it = 0; it < iters && nc > 0; it++) {
                vec3 F = v3(0, 0, 0), Tq = v3(0, 0, 0);
                for (int k = 0; k < nc; k++) {
                    F = vadd(F, ct[k].c.lam);
                    Tq = vadd(Tq, vcross(ct[k].c.r, ct[k].c.lam));
                }
                vec3 vi = vadd(v_pred, vscale(F, 1.0 / m));
                vec3 wi = vadd(w_pred, mvmul(W, Tq));
                pd_joint_vel(ct, nc, qd_star, M, D, qd);
                for (int k = 0; k < nc; k++) {
                    contact_t *c = &ct[k].c;
                    vec3 u = vsub(vadd(vi, vcross(wi, c->r)), pd_link_vel(&ct[k], qd));
                    vec3 lproj = contact_update(c->lam, u, c->n, c->b, c->inv_kn, c->inv_kt, mu);
                    c->lam_next = vadd(c->lam, vscale(vsub(lproj, c->lam), 1.0 / nc));
                }
                for (int k = 0; k < nc; k++) ct[k].c.lam = ct[k].c.lam_next;
                diag[5] += 1;
            }
            vec3 F = v3(0, 0, 0), Tq = v3(0, 0, 0);
            for (int k = 0; k < nc; k++) {
                F = vadd(F, ct[k].c.lam);
                Tq = vadd(Tq, vcross(ct[k].c.r, ct[k].c.lam));
            }
            v = vadd(v_pred, vscale(F, 1.0 / m));
            w = vadd(w_pred, mvmul(W, Tq));
            pd_joint_vel(ct, nc, qd_star, M, D, qd);

            x = vadd(x, vscale(v, h));
            q = qnormalize(qmul(quat_exp(vscale(w, h)), q));
            for (int a = 0; a < D; a++) {
                qdj[a] = qd[a];
                qj[a] += h * qd[a];
            }

            for (int k = 0; k < nc; k++) {
                const contact_t *c = &ct[k].c;
                if (c->pad < 0) continue;
                double *fp = forces + 3 * c->pad;
                fp[0] -= c->lam.x / h; fp[1] -= c->lam.y / h; fp[2] -= c->lam.z / h;
                double ln = vdot(c->lam, c->n);
                if (!(ln > 0)) continue;
                vec3 vrel = vsub(vadd(v, vcross(w, c->r)), pd_link_vel(&ct[k], qd));
                vec3 vt = vsub(vrel, vscale(c->n, vdot(vrel, c->n)));
                vec3 wl = v3(0, 0, 0);
                for (int a = 0; a < ct[k].nj; a++) wl = vadd(wl, vscale(JF[ct[k].j0 + a].z, qd[ct[k].j0 + a]));
                double spin = vdot(vsub(w, wl), c->n);
                double *A = acc + 8 * c->pad;
                A[0] += ln;
                A[1] += ln * vt.x; A[2] += ln * vt.y; A[3] += ln * vt.z;
                A[4] += ln * c->n.x; A[5] += ln * c->n.y; A[6] += ln * c->n.z;
                A[7] += ln * spin;
            }
            if (last_n) {   /* the last substep's contacts: link, point, impulse */
                int nk = nc < last_cap ? nc : last_cap;
                for (int k = 0; k < nk; k++) {
                    double *o = last_ct + 7 * k;
                    o[0] = ct[k].c.id >> 8;
                    o[1] = ct[k].p.x; o[2] = ct[k].p.y; o[3] = ct[k].p.z;
                    o[4] = ct[k].c.lam.x; o[5] = ct[k].c.lam.y; o[6] = ct[k].c.lam.z;
                }
                *last_n = nk;
            }
        }
        pose7[0] = x.x; pose7[1] = x.y; pose7[2] = x.z;
        pose7[3] = q.w; pose7[4] = q.x; pose7[5] = q.y; pose7[6] = q.z;
        vel6[0] = v.x; vel6[1] = v.y; vel6[2] = v.z; vel6[3] = w.x; vel6[4] = w.y; vel6[5] = w.z;
        int finite = 1;
        for (int k = 0; k < 7; k++) finite &= isfinite(pose7[k]);
        for (int k = 0; k < 6; k++) finite &= isfinite(vel6[k]);
        for (int a = 0; a < D; a++) finite &= isfinite(qj[a]) && isfinite(qdj[a]);
        if (!finite) *status |= ORC_NONFINITE;
        else if (vnorm(x) > cfg->escape_radius) *status |= ORC_ESCAPED;
    }
    for (int k = 0; k < 3 * P; k++) forces[k] /= ns;

    /* the hand's sensors at the end of the frame */
    orc_fk(sc, qj, lp);
    for (int l = 0; l < P; l++) {
        pad_pose_of(sc, l, lp, pad_pose + 7 * l);
        const double *A = acc + 8 * l;
        if (!(A[0] > 0)) continue;
        vec3 vt = vscale(v3(A[1], A[2], A[3]), 1.0 / A[0]);
        vec3 nb = v3(A[4], A[5], A[6]);
        nb = vscale(nb, 1.0 / vnorm(nb));
        double spin = A[7] / A[0];
        slip_mag[2 * l] = vnorm(vt);
        slip_mag[2 * l + 1] = spin;
        int flags = 0;
        if (vnorm(vt) > pd->v_slip) {
            pose_t Lk = pose_from7(lp + 7 * sc->pad_link[l]);
            vec3 ax = v3(Lk.R.m[0][0], Lk.R.m[1][0], Lk.R.m[2][0]);
            vec3 e1 = vsub(ax, vscale(nb, vdot(ax, nb)));
            e1 = vscale(e1, 1.0 / vnorm(e1));
            vec3 e2 = vcross(nb, e1);
            double d1 = vdot(vt, e1), d2 = vdot(vt, e2), dn = sqrt(d1 * d1 + d2 * d2);
            slip_d[2 * l] = d1 / dn; slip_d[2 * l + 1] = d2 / dn;
            flags |= 1;
        }
        if (fabs(spin) > pd->w_slip) {
            flags |= 2;
            if (spin > 0) flags |= 4;
        }
        slip_flags[l] = flags;
    }
    free(lp); free(JF); free(qd_star); free(qd); free(acc);
}

/*
 * Advance N environments with the PD-driven hand over n_frames frames. qj, qdj
 * [N][D] are the joint positions and velocities (in/out). Outputs of the last
 * frame: forces [N][P][3], pad_pose [N][P][7], slip_d [N][P][2], slip_flags
 * [N][P] (bit 0 translational slip, bit 1 rotational slip, bit 2 spin > 0),
 * slip_mag [N][P][2] (mean relative tangential speed, mean relative spin;
 * zero for a pad without contact), diag [N][ORC_DIAG]; with last_n non-NULL, the last substep's contacts
 * last_ct [N][last_cap][7] (link, world point, impulse on the object) and
 * their count last_n [N].
 */
int orc_step_pd(const orc_scene *sc, const orc_config *cfg, const orc_pd *pd, int N, const double *q_traj,
                int frame0, int n_frames, double *pose, double *vel, const double *theta, const int32_t *shape,
                const int32_t *iters, int32_t *status, double *qj, double *qdj, double *forces,
                double *pad_pose, double *slip_d, int32_t *slip_flags, double *slip_mag, double *diag,
                double *last_ct, int32_t *last_n, int last_cap) {
    const int D = 4 * sc->n_fingers, n_links = 1 + 4 * sc->n_fingers, ns = cfg->substeps;
    const int P = sc->n_pads;
    double *u_all = (double *)malloc(sizeof(double) * (D > 0 ? D : 1) * (ns + 1));
    int cap = 1;
    for (int s = 0; s < sc->n_shapes; s++) cap = cap > sc->shape_count[s] ? cap : sc->shape_count[s];
    cap = cap * n_links + 1;
    pd_contact_t *ct = (pd_contact_t *)malloc(sizeof(pd_contact_t) * cap);
    for (int f = frame0; f < frame0 + n_frames; f++) {
        for (int k = 0; k <= ns; k++)
            for (int j = 0; j < D; j++) {
                double q0 = q_traj[(size_t)f * D + j], q1 = q_traj[(size_t)(f + 1) * D + j];
                u_all[(size_t)k * D + j] = q0 + ((double)k / ns) * (q1 - q0);
            }
        for (int i = 0; i < N; i++) {
            int it = iters ? iters[i] : cfg->iters;
            step_env_pd(sc, cfg, pd, u_all, ns, pose + 7 * (size_t)i, vel + 6 * (size_t)i,
                        theta + 2 * (size_t)i, shape ? shape[i] : 0, it, status + i, qj + (size_t)i * D,
                        qdj + (size_t)i * D, forces + (size_t)i * 3 * P, pad_pose + (size_t)i * 7 * P,
                        slip_d + (size_t)i * 2 * P, slip_flags + (size_t)i * P, slip_mag + (size_t)i * 2 * P,
                        diag + (size_t)i * ORC_DIAG, ct, cap, last_n ? last_ct + (size_t)i * 7 * last_cap : NULL, last_n ? last_n + i : NULL,
                        last_cap);
        }
    }
    free(u_all); free(ct);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* the full cost of Sec. III-C over the PD hand's observation                 */
/* ------------------------------------------------------------------------- */
/*
 * C = w1 |q - q_gt| + sum_l [ w2 |P - P_gt| + w3 |angle(R^-1 R_gt)|
 *       + w4 (1 - alpha) + alpha (w5 | |c| - |c_gt| | + w6 angle(c, c_gt))
 *       + w7 (1 - beta) + beta w8 angle(d, d_gt)
 *       + w9 (1 - gamma) + gamma w10 |r - r_gt| ]
 * alpha, beta, gamma = 1 when the two agree on contact (|c| > tau), on
 * translational slip and on rotational slip. Angles between force vectors
 * count only when both pads are in contact, between slip directions only
 * when both slip, and |r - r_gt| only when both slip rotationally (the angle
 * or direction of an absent contact or slip is undefined).
 */
static double vangle(vec3 a, vec3 b) { return atan2(vnorm(vcross(a, b)), vdot(a, b)); }

static double frame_cost_full(const double *wt, double tau, int D, int P, const double *q_a, const double *q_b,
                              const double *pp_a, const double *pp_b, const double *c_a, const double *c_b,
                              const double *d_a, const double *d_b, const int32_t *f_a, const int32_t *f_b) {
    double dq = 0;
    for (int j = 0; j < D; j++) dq += (q_a[j] - q_b[j]) * (q_a[j] - q_b[j]);
    double cost = wt[0] * sqrt(dq);
    for (int l = 0; l < P; l++) {
        const double *pa = pp_a + 7 * l, *pb = pp_b + 7 * l;
        cost += wt[1] * vnorm(v3(pa[0] - pb[0], pa[1] - pb[1], pa[2] - pb[2]));
        quat qa = {pa[3], pa[4], pa[5], pa[6]}, qb = {pb[3], pb[4], pb[5], pb[6]};
        quat rel = qmul(qconj(qa), qb);
        cost += wt[2] * 2.0 * atan2(vnorm(v3(rel.x, rel.y, rel.z)), fabs(rel.w));
        vec3 ca = v3(c_a[3 * l], c_a[3 * l + 1], c_a[3 * l + 2]), cb = v3(c_b[3 * l], c_b[3 * l + 1], c_b[3 * l + 2]);
        double ma = vnorm(ca), mb = vnorm(cb);
        int in_a = ma > tau, in_b = mb > tau;
        if (in_a != in_b) {
            cost += wt[3];
        } else {
            cost += wt[4] * fabs(ma - mb);
            if (in_a) cost += wt[5] * vangle(ca, cb);
        }
        int ta = f_a[l] & 1, tb = f_b[l] & 1;
        if (ta != tb) {
            cost += wt[6];
        } else if (ta) {
            const double *da = d_a + 2 * l, *db = d_b + 2 * l;
            cost += wt[7] * atan2(fabs(da[0] * db[1] - da[1] * db[0]), da[0] * db[0] + da[1] * db[1]);
        }
        int ra = (f_a[l] >> 1) & 1, rb = (f_b[l] >> 1) & 1;
        if (ra != rb) {
            cost += wt[8];
        } else if (ra) {
            cost += wt[9] * fabs((double)((f_a[l] >> 2) & 1) - (double)((f_b[l] >> 2) & 1));
        }
    }
    return cost;
}

/* running window mean and argmin of the full cost, as orc_cost */
int orc_cost_full(const double *wt, double tau, int N, int D, int P, const double *qj, const double *pad_pose,
                  const double *forces, const double *slip_d, const int32_t *slip_flags, const double *g_q,
                  const double *g_pose, const double *g_forces, const double *g_d, const int32_t *g_flags,
                  const int32_t *status, double *c_sum, int n_window, double *c_mean, double *cost_out) {
    int best = 0;
    double best_c = INFINITY;
    for (int i = 0; i < N; i++) {
        double c = (status[i] & ORC_DIVERGED)
                       ? INFINITY
                       : frame_cost_full(wt, tau, D, P, qj + (size_t)D * i, g_q, pad_pose + (size_t)7 * P * i, g_pose,
                                         forces + (size_t)3 * P * i, g_forces, slip_d + (size_t)2 * P * i, g_d,
                                         slip_flags + (size_t)P * i, g_flags);
        if (cost_out) cost_out[i] = c;
        c_sum[i] += c;
        double cm = c_sum[i] / n_window;
        if (c_mean) c_mean[i] = cm;
        if (isnan(cm)) cm = INFINITY;
        if (cm < best_c || (i == 0)) { best_c = cm; best = i; }
    }
    return best;
}
