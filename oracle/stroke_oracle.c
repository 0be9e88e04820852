/*
 * FP64 CPU oracle for GPU-friendly stroke expansion
 * (R. Levien and A. Uguray, "GPU-friendly Stroke Expansion", arXiv 2405.00127).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It is a plain, slow,
 * double-precision restatement of the paper's method and shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What is computed (per stroked path, in output order):
 *   - decode of SVG-style verbs into subpaths (Section 8.1: moveto/lineto/
 *     curveto/closepath), dropping zero-length segments and inserting the
 *     closing line of closed subpaths (Section 8.2);
 *   - optional dashing of each subpath into open dash subpaths (SVG dash
 *     semantics; the paper dashes on the CPU, Section 9.3);
 *   - per segment: cubic -> Euler-spiral (ES) adaptive subdivision with the
 *     two-word recursion stack (Algorithm 2, Section 7), the closed-form error
 *     prediction (Section 7.1), geometric Hermite interpolation (Appendix A),
 *     derivative re-sampling at input cusps (Section 7.3);
 *   - per ES piece and side: parallel-curve flattening with the subdivision
 *     density integral and its piecewise approximation (Sections 4.1, 4.2) or
 *     arc approximation (Section 5), split at the parallel-curve cusp
 *     (Section 7.3.1) with evolute patches emitted twice (Section 6);
 *   - joins (bevel/miter/round, outer contour plus inner contour through the
 *     joint) and caps (butt/square/round) with SVG semantics (Section 8.1,
 *     Algorithm 1), round shapes flattened with the exact arc metric
 *     (Section 2.1).
 *
 * Every decision that turns floating point into an integer records its
 * relative distance to the decision boundary ("margin"); the tests treat a
 * segment whose smallest margin is tiny as having several correct answers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* small vector helpers                                               */
/* ------------------------------------------------------------------ */
typedef struct { double x, y; } V2;

static V2 vec(double x, double y) { V2 r; r.x = x; r.y = y; return r; }
static V2 vadd(V2 a, V2 b) { return vec(a.x + b.x, a.y + b.y); }
static V2 vsub(V2 a, V2 b) { return vec(a.x - b.x, a.y - b.y); }
static V2 vmul(V2 a, double s) { return vec(a.x * s, a.y * s); }
static double vdot(V2 a, V2 b) { return a.x * b.x + a.y * b.y; }
static double vcross(V2 a, V2 b) { return a.x * b.y - a.y * b.x; }
static double vlen(V2 a) { return hypot(a.x, a.y); }
static V2 cmul(V2 a, V2 b) { return vec(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
static V2 cdiv(V2 a, V2 b) {
    double d = b.x * b.x + b.y * b.y;
    return vec((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
static V2 vrot(V2 a, double ang) {
    double c = cos(ang), s = sin(ang);
    return vec(a.x * c - a.y * s, a.x * s + a.y * c);
}
static int veq(V2 a, V2 b) { return a.x == b.x && a.y == b.y; }

/* ------------------------------------------------------------------ */
/* Section 4.1: subdivision density integral of the ES parallel curve  */
/* f(x) = int_0^x sqrt|u^2 - 1| du, odd.  For x >= 1 the pi/4 constant  */
/* sits outside the 1/2 factor (the only placement that keeps f         */
/* continuous at x = 1, where f(1) = pi/4).                             */
/* ------------------------------------------------------------------ */
double orc_f_exact(double x) {
    double a = fabs(x), r;
    if (a <= 1.0) r = 0.5 * (a * sqrt(1.0 - a * a) + asin(a));
    else r = 0.5 * (a * sqrt(a * a - 1.0) - acosh(a)) + ORC_PI / 4.0;
    return copysign(r, x);
}

/* Section 4.2: piecewise, invertible approximation of f.  On [0.8, 1.25)
 * the power (x - 1)^1.5 is read as (x - 1)|x - 1|^0.5, which is the reading
 * that makes the pieces meet at 0.8. */
static const double FA_C1 = 1.0976991822760038;
static const double FA_C2 = 0.9148117935952064;
static const double FA_C3 = 0.16145779359520596;

static double fa_pos(double a) {
    if (a < 0.8) return sin(FA_C1 * a) / FA_C1;
    if (a < 1.25) {
        double e = a - 1.0;
        return sqrt(8.0) / 3.0 * e * sqrt(fabs(e)) + ORC_PI / 4.0;
    }
    if (a < 2.1) return 0.6406 * a * a - 0.81 * a + FA_C2;
    return 0.5 * a * a - 0.156 * a + FA_C3;
}

double orc_f_approx(double x) { return copysign(fa_pos(fabs(x)), x); }

/* derivative of the approximation, piece by piece */
double orc_f_approx_deriv(double x) {
    double a = fabs(x);
    if (a < 0.8) return cos(FA_C1 * a);
    if (a < 1.25) return sqrt(2.0) * sqrt(fabs(a - 1.0));
    if (a < 2.1) return 2.0 * 0.6406 * a - 0.81;
    return a - 0.156;
}

/* exact inverse of the approximation, piece by piece */
double orc_f_approx_inv(double y) {
    double a = fabs(y), x;
    double y08 = fa_pos(0.8), y125 = fa_pos(1.25), y21 = fa_pos(2.1);
    if (a < y08) {
        x = asin(FA_C1 * a) / FA_C1;
    } else if (a < y125) {
        double v = (a - ORC_PI / 4.0) * 3.0 / sqrt(8.0);
        x = 1.0 + copysign(pow(fabs(v), 2.0 / 3.0), v);
    } else if (a < y21) {
        /* 0.6406 x^2 - 0.81 x + (c2 - a) = 0, larger root */
        double A = 0.6406, B = -0.81, Cc = FA_C2 - a;
        x = (-B + sqrt(B * B - 4.0 * A * Cc)) / (2.0 * A);
    } else {
        double A = 0.5, B = -0.156, Cc = FA_C3 - a;
        x = (-B + sqrt(B * B - 4.0 * A * Cc)) / (2.0 * A);
    }
    return copysign(x, y);
}

/* ------------------------------------------------------------------ */
/* Appendix A: geometric Hermite interpolation polynomials.            */
/* k = theta0 + theta1, delta = theta1 - theta0.  Curvature of the unit */
/* ES is k0 + k1 (s - 1/2) on s in [0, 1] (centred reading: the only    */
/* one under which k0 = theta0 + theta1 holds).                         */
/* ------------------------------------------------------------------ */
void orc_gh(double k, double d, double* k1_out, double* c_out) {
    double d2 = d * d, k2 = k * k;
    double k1 = 6.0 * d
        - d * d2 / 70.0
        - d * d2 * d2 / 10780.0
        + d * d2 * d2 * d2 * 2.769178184818219e-7
        - k2 * d / 10.0
        + k2 * d * d2 / 4200.0
        + k2 * d * d2 * d2 * 1.6959677820260655e-5
        - k2 * k2 * d / 1400.0
        + k2 * k2 * d * d2 * 6.84915970574303e-5
        - k2 * k2 * k2 * d * 7.936475029053326e-6;
    double c = 1.0
        - d2 / 40.0
        + d2 * d2 * 0.00034226190482569864
        - d2 * d2 * d2 * 1.9349474568904524e-6
        - k2 / 24.0
        + k2 * d2 * 0.0024702380951963226
        - k2 * d2 * d2 * 3.7297408997537985e-5
        + k2 * k2 / 1920.0
        - k2 * k2 * d2 * 4.87350869747975e-5
        - k2 * k2 * k2 * 3.1001936068463107e-6;
    *k1_out = k1;
    *c_out = c;
}

/* ------------------------------------------------------------------ */
/* Section 7.1: error prediction of the cubic -> ES fit.              */
/* p0, p1: endpoints; q0, q1: derivatives dB/dt there; dt: parameter   */
/* length of the sub-cubic.  Angles: the start tangent lies at -theta0 */
/* and the end tangent at +theta1 relative to the chord.               */
/* out: theta0, theta1, chord length, error (in the units of the input) */
/* ------------------------------------------------------------------ */
static double es_area(double d0, double d1, double t0, double t1) {
    return 0.15 * (2.0 * d0 * sin(t0) + 2.0 * d1 * sin(t1) - d0 * d1 * sin(t0 + t1));
}

/* exported for the tests */
double orc_cubic_area(double d0, double d1, double t0, double t1) { return es_area(d0, d1, t0, t1); }

void orc_fit(const double* p0, const double* p1, const double* q0, const double* q1, double dt,
             double* out) {
    V2 P0 = vec(p0[0], p0[1]), P1 = vec(p1[0], p1[1]);
    V2 Q0 = vec(q0[0], q0[1]), Q1 = vec(q1[0], q1[1]);
    V2 ch = vsub(P1, P0);
    double cl = vlen(ch);
    if (cl == 0.0) {
        out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; out[3] = INFINITY;
        return;
    }
    double th0 = atan2(vcross(Q0, ch), vdot(Q0, ch));
    double th1 = atan2(vcross(ch, Q1), vdot(ch, Q1));
    double d0 = vlen(Q0) * dt / (3.0 * cl);
    double d1 = vlen(Q1) * dt / (3.0 * cl);
    double den0 = 1.0 + cos(th0), den1 = 1.0 + cos(th1);
    double err;
    if (!(den0 > 0.0) || !(den1 > 0.0)) {
        err = INFINITY;
    } else {
        double db0 = 2.0 / (3.0 * den0), db1 = 2.0 / (3.0 * den1);
        double k = th0 + th1, dd = th0 - th1;
        double e1 = 4.6255e-6 * pow(fabs(k), 5.0) + 7.5e-3 * k * k * fabs(dd);
        double e2 = 1.55 * fabs(es_area(d0, d1, th0, th1) - es_area(db0, db1, th0, th1));
        double e3 = (0.005 * fabs(k) + 0.07 * fabs(dd)) * sqrt((db0 - d0) * (db0 - d0) + (db1 - d1) * (db1 - d1));
        err = (e1 + e2 + e3) * cl;
    }
    out[0] = th0; out[1] = th1; out[2] = cl; out[3] = err;
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes (16 points), computed once by Newton iteration */
/* on the Legendre polynomial.                                         */
/* ------------------------------------------------------------------ */
#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];

static void legendre(int n, double x, double* p, double* dp) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

__attribute__((constructor)) static void gl_init(void) {
    for (int i = 0; i < GL_N; i++) {
        double x = cos(ORC_PI * (i + 0.75) / (GL_N + 0.5)), p, dp;
        for (int it = 0; it < 100; it++) {
            legendre(GL_N, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        legendre(GL_N, x, &p, &dp);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* ------------------------------------------------------------------ */
/* Euler-spiral piece                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    V2 p0, p1, q0, q1;   /* endpoints and sampled derivatives */
    double th0, th1;     /* fit angles */
    double k0, k1, c;    /* Appendix A parameters of the unit ES */
    double L;            /* arc length = chord / c */
    double chord_len;
    double t0, t1;       /* source parameter range */
    V2 rot;              /* complex factor mapping the unit ES onto the chord */
    int degenerate;      /* zero chord (only when forced at the depth cap) */
} ES;

/* tangent angle of the unit ES at s in [0, 1] */
static double es_theta(const ES* e, double s) {
    return -e->th0 + e->k0 * s + 0.5 * e->k1 * (s * s - s);
}

/* position on the unit ES: int_0^s exp(i theta) ds, composite 16-point GL */
static V2 es_unit_pos(const ES* e, double s) {
    if (s == 0.0) return vec(0.0, 0.0);
    double A = (fabs(e->k0) + fabs(e->k1)) * fabs(s);
    int m = 1 + (int)A;
    double h = s / m;
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < m; j++) {
        double base = j * h;
        for (int i = 0; i < GL_N; i++) {
            double sg = base + 0.5 * h * (gl_x[i] + 1.0);
            double th = es_theta(e, sg);
            ax += gl_w[i] * cos(th);
            ay += gl_w[i] * sin(th);
        }
    }
    return vec(0.5 * h * ax, 0.5 * h * ay);
}

/* exported for the tests: unit-ES position for given (theta0, theta1) */
void orc_es_unit_point(double th0, double th1, double s, double* out) {
    ES e;
    memset(&e, 0, sizeof e);
    e.th0 = th0; e.th1 = th1; e.k0 = th0 + th1;
    orc_gh(e.k0, th1 - th0, &e.k1, &e.c);
    V2 p = es_unit_pos(&e, s);
    out[0] = p.x; out[1] = p.y;
}

static const double C_MIN = 0.25;   /* smallest accepted GH chord/arc ratio */

/* Appendix A: the unit ES is scaled, rotated and translated so that its ends
 * land on the chord.  The arc length is taken from the same quadrature that
 * places the curve (|P(1)| rather than the polynomial c, which agree to 1e-5
 * for |theta| <= 1), so curvature, evolute and counts all describe the curve
 * whose points are emitted.  |P(1)| is floored at 0.05 for pieces forced at
 * the depth cap. */
static void es_setup(ES* e) {
    e->k0 = e->th0 + e->th1;
    orc_gh(e->k0, e->th1 - e->th0, &e->k1, &e->c);
    V2 u1 = es_unit_pos(e, 1.0);
    double m = vlen(u1);
    e->L = e->chord_len / (m > 0.05 ? m : 0.05);
    e->rot = cdiv(vsub(e->p1, e->p0), u1);
}

/* normalised curvature (per unit ES length) */
static double es_kn(const ES* e, double s) { return e->k0 + e->k1 * (s - 0.5); }

static V2 es_pos(const ES* e, double s) { return vadd(e->p0, cmul(es_unit_pos(e, s), e->rot)); }

static V2 es_tangent(const ES* e, double s) {
    double th = es_theta(e, s);
    V2 t = cmul(vec(cos(th), sin(th)), e->rot);
    return vmul(t, 1.0 / vlen(t));
}

/* The one formula for every offset point at a sampled (point, derivative)
 * pair: P + sh * unit right normal of q.  Segment ends, joins and caps all
 * use it, so points shared between them coincide exactly. */
static V2 shared_offset(V2 P, V2 q, double sh) {
    double l = vlen(q);
    return vec(P.x + sh * (q.y / l), P.y + sh * (-q.x / l));
}

static V2 es_offset(const ES* e, double s, double sh) {
    if (s == 0.0) return shared_offset(e->p0, e->q0, sh);
    if (s == 1.0) return shared_offset(e->p1, e->q1, sh);
    V2 T = es_tangent(e, s);
    return vadd(es_pos(e, s), vec(sh * T.y, -sh * T.x));
}

/* centre of curvature: position + left normal / curvature */
static V2 es_evolute(const ES* e, double s) {
    V2 T = es_tangent(e, s);
    double kappa = es_kn(e, s) / e->L;
    return vadd(es_pos(e, s), vmul(vec(-T.y, T.x), 1.0 / kappa));
}

/* ------------------------------------------------------------------ */
/* Configuration, result buffers                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    double tol_fit, tol_flat;
    int arcs;
    int refine;  /* line output: exact density integral and Newton-refined inverse (Section 4.2) */
    int max_depth;
    double deriv_eps, deriv_dt;
    int64_t max_count;
} Cfg;

#define PIECE_STRIDE 21

typedef struct orc_result {
    int64_t n_seg, n_prim, n_piece;
    int32_t* seg_kind;        /* 0 segment, 1 closing line, 2 marker, 3 empty path */
    int32_t* seg_path;
    int64_t* seg_first_prim;
    int64_t* seg_count;
    double* seg_margin;
    int32_t* seg_npiece;
    double* seg_dash_margin;  /* per record: its path's smallest relative dash-cut margin (INFINITY if solid) */
    double* prim;             /* n_prim x 5: x0 y0 x1 y1 curvature */
    int8_t* prim_kind;
    int8_t* prim_side;
    int32_t* prim_piece;
    double* prim_cond;        /* FP32 conditioning of each primitive's geometry (see Em.cond) */
    double* piece;            /* n_piece x PIECE_STRIDE */
    int32_t* piece_seg;
    int64_t cap_seg, cap_prim, cap_piece;
    int32_t error;            /* 0 ok, 1 count cap hit, 2 bad input */
    /* why a segment is fragile, kept apart so each widening of the plain 1e-4
     * rule can be counted: */
    double* seg_raw_margin;   /* smallest relative decision margin, not scaled by the FP32 conditioning */
    int8_t* seg_sens;         /* 1: moving a piece's fit angles by their FP32 uncertainty changes its count */
    /* work counters (units of the arithmetic roofline): cubic -> Euler-spiral fit
     * attempts of Algorithm 2, and output vertices (every chain of primitives
     * has one vertex more than primitives) */
    int64_t n_fit, n_vert;
} orc_result;

enum { PK_OFFSET = 0, PK_OFFSET_REV = 1, PK_EVOLUTE = 2, PK_CONNECT = 3, PK_JOIN_OUTER = 4,
       PK_JOIN_INNER = 5, PK_CAP = 6, PK_DEGEN = 7 };

static void* grow(void* p, int64_t n, size_t elem) { return realloc(p, (size_t)n * elem); }

static void res_push_seg(orc_result* r, int kind, int path) {
    if (r->n_seg == r->cap_seg) {
        r->cap_seg = r->cap_seg ? 2 * r->cap_seg : 1024;
        r->seg_kind = grow(r->seg_kind, r->cap_seg, 4);
        r->seg_path = grow(r->seg_path, r->cap_seg, 4);
        r->seg_first_prim = grow(r->seg_first_prim, r->cap_seg, 8);
        r->seg_count = grow(r->seg_count, r->cap_seg, 8);
        r->seg_margin = grow(r->seg_margin, r->cap_seg, 8);
        r->seg_npiece = grow(r->seg_npiece, r->cap_seg, 4);
        r->seg_dash_margin = grow(r->seg_dash_margin, r->cap_seg, 8);
        r->seg_raw_margin = grow(r->seg_raw_margin, r->cap_seg, 8);
        r->seg_sens = grow(r->seg_sens, r->cap_seg, 1);
    }
    int64_t i = r->n_seg++;
    r->seg_kind[i] = kind;
    r->seg_path[i] = path;
    r->seg_first_prim[i] = r->n_prim;
    r->seg_count[i] = 0;
    r->seg_margin[i] = INFINITY;
    r->seg_npiece[i] = 0;
    r->seg_dash_margin[i] = INFINITY;
    r->seg_raw_margin[i] = INFINITY;
    r->seg_sens[i] = 0;
}

typedef struct {
    orc_result* r;
    const Cfg* cfg;
    int flip;           /* emit each primitive reversed (the -h side) */
    int side;
    int32_t piece;
    double margin;
    double raw_margin;  /* the same without the FP32-conditioning scale */
    int sens;           /* the count-sensitivity test fired */
    double cond;        /* FP32 relative error estimate of the current decision's inputs */
    double dash_margin; /* smallest dash-cut margin of the current path */
    double pcond;       /* when >= 0: conditioning recorded with emitted primitives instead of cond */
    V2 chain_end;       /* the previous primitive's end, before any flip (vertex counting) */
    int chain_open;
} Em;

/* FP32 unit roundoff; the method's arithmetic is FP32 (Section 1) */
static const double EPS32 = 5.9604644775390625e-08;

/* Record a decision's relative distance to its boundary.  A decision whose
 * inputs carry an FP32 relative error of `cond` cannot be resolved closer than
 * ~8 cond, so its margin is reported relative to max(1e-4, 8 cond): the
 * segment counts as fragile (several answers correct) exactly when the margin
 * falls below max(1e-4, 8 cond). */
static void upd(Em* em, double m) {
    if (m < em->raw_margin) em->raw_margin = m;
    double scale = 8.0 * em->cond / 1e-4;
    if (scale > 1.0) m /= scale;
    if (m < em->margin) em->margin = m;
}


static void emit(Em* em, V2 a, V2 b, double k, int kind) {
    orc_result* r = em->r;
    if (r->n_prim == r->cap_prim) {
        r->cap_prim = r->cap_prim ? 2 * r->cap_prim : 4096;
        r->prim = grow(r->prim, r->cap_prim * 5, 8);
        r->prim_kind = grow(r->prim_kind, r->cap_prim, 1);
        r->prim_side = grow(r->prim_side, r->cap_prim, 1);
        r->prim_piece = grow(r->prim_piece, r->cap_prim, 4);
        r->prim_cond = grow(r->prim_cond, r->cap_prim, 8);
    }
    /* a primitive continuing the previous one's chain adds one vertex, else two */
    r->n_vert += (em->chain_open && veq(a, em->chain_end)) ? 1 : 2;
    em->chain_end = b;
    em->chain_open = 1;
    if (em->flip) { V2 t = a; a = b; b = t; k = -k; }
    int64_t i = r->n_prim++;
    double* p = r->prim + 5 * i;
    p[0] = a.x; p[1] = a.y; p[2] = b.x; p[3] = b.y; p[4] = k;
    r->prim_kind[i] = (int8_t)kind;
    r->prim_side[i] = (int8_t)em->side;
    r->prim_piece[i] = em->piece;
    r->prim_cond[i] = em->pcond >= 0.0 ? em->pcond : em->cond;
}

static int32_t push_piece(orc_result* r, const ES* e, int64_t seg, double em_cond_of_piece) {
    if (r->n_piece == r->cap_piece) {
        r->cap_piece = r->cap_piece ? 2 * r->cap_piece : 1024;
        r->piece = grow(r->piece, r->cap_piece * PIECE_STRIDE, 8);
        r->piece_seg = grow(r->piece_seg, r->cap_piece, 4);
    }
    int64_t i = r->n_piece++;
    double* d = r->piece + PIECE_STRIDE * i;
    d[0] = e->t0; d[1] = e->t1;
    d[2] = e->p0.x; d[3] = e->p0.y; d[4] = e->p1.x; d[5] = e->p1.y;
    d[6] = e->q0.x; d[7] = e->q0.y; d[8] = e->q1.x; d[9] = e->q1.y;
    d[10] = e->th0; d[11] = e->th1; d[12] = e->k0; d[13] = e->k1; d[14] = e->c; d[15] = e->L;
    d[16] = e->rot.x; d[17] = e->rot.y; d[18] = e->chord_len; d[19] = e->degenerate;
    d[20] = em_cond_of_piece;
    r->piece_seg[i] = (int32_t)seg;
    return (int32_t)i;
}

/* ceil with the max(1, .) floor used for every count; records the margin */
static int64_t count_of(Em* em, double N) {
    double m;
    if (!(N == N)) N = 1.0;
    if (N <= 1.0) m = 1.0 - N;
    else m = fmin(N - floor(N), ceil(N) - N) / N;
    upd(em, m);
    double c = ceil(N);
    if (c < 1.0) c = 1.0;
    if (c > (double)em->cfg->max_count) {
        em->r->error = 1;
        c = (double)em->cfg->max_count;
    }
    return (int64_t)c;
}

/* ------------------------------------------------------------------ */
/* Flattening counts and sample positions                              */
/* ------------------------------------------------------------------ */

/* divided difference of f_approx over [ua, ub].  The difference quotient is
 * used whenever the F difference is resolved in double precision; only a
 * vanishing difference falls back to the derivative at the midpoint. */
static int f_diff_resolved(double ua, double ub) {
    double Fa = orc_f_approx(ua), Fb = orc_f_approx(ub);
    return ub != ua && fabs(Fb - Fa) > 1e-10 * fmax(1.0, fabs(Fa));
}

static double dd_f(double ua, double ub) {
    if (f_diff_resolved(ua, ub)) return (orc_f_approx(ub) - orc_f_approx(ua)) / (ub - ua);
    return orc_f_approx_deriv(0.5 * (ua + ub));
}

/* Section 4.1: number of lines for the parallel curve at signed normalised
 * offset sh_n (= sigma h / L) over the unit-ES range [a, b].  With
 * u(s) = -1 - 2 sh_n kappa_n(s) the inflection maps to -1 and the offset
 * cusp to +1; the density integral is |F(ub) - F(ua)| / (4 h_n^1.5 |k1|),
 * written as (b - a) * divided-difference / (2 sqrt(h_n)) so that the
 * constant-curvature limit k1 -> 0 stays finite. */
double orc_line_count(double k0, double k1, double sh_n, double a, double b, double tol_n) {
    double ka = k0 + k1 * (a - 0.5), kb = k0 + k1 * (b - 0.5);
    double ua = -1.0 - 2.0 * sh_n * ka, ub = -1.0 - 2.0 * sh_n * kb;
    double I = (b - a) * dd_f(ua, ub) / (2.0 * sqrt(fabs(sh_n)));
    return fabs(I) / sqrt(8.0 * tol_n);
}

static double line_s(const ES* e, double sh_n, double a, double b, int64_t i, int64_t n) {
    if (i == 0) return a;
    if (i == n) return b;
    double ua = -1.0 - 2.0 * sh_n * es_kn(e, a), ub = -1.0 - 2.0 * sh_n * es_kn(e, b);
    double d = ub - ua;
    double fr = (double)i / (double)n;
    if (!f_diff_resolved(ua, ub)) return a + (b - a) * fr;
    double Fa = orc_f_approx(ua), Fb = orc_f_approx(ub);
    double ui = orc_f_approx_inv(Fa + (Fb - Fa) * fr);
    return a + (b - a) * ((ui - ua) / d);
}

/* Refined mode (Section 4.2): the count takes the exact integral f of
 * Section 4.1 instead of its approximation, and each vertex solves
 * f(u) = target by two Newton steps from the approximation's inverse.
 * f' = sqrt|u^2 - 1| (the subdivision density itself). */
double orc_f_exact_deriv(double x) { return sqrt(fabs(x * x - 1.0)); }

static int fx_diff_resolved(double ua, double ub) {
    double Fa = orc_f_exact(ua), Fb = orc_f_exact(ub);
    return ub != ua && fabs(Fb - Fa) > 1e-10 * fmax(1.0, fabs(Fa));
}

static double dd_fx(double ua, double ub) {
    if (fx_diff_resolved(ua, ub)) return (orc_f_exact(ub) - orc_f_exact(ua)) / (ub - ua);
    return orc_f_exact_deriv(0.5 * (ua + ub));
}

/* orc_line_count with the exact integral */
double orc_line_count_exact(double k0, double k1, double sh_n, double a, double b, double tol_n) {
    double ka = k0 + k1 * (a - 0.5), kb = k0 + k1 * (b - 0.5);
    double ua = -1.0 - 2.0 * sh_n * ka, ub = -1.0 - 2.0 * sh_n * kb;
    double I = (b - a) * dd_fx(ua, ub) / (2.0 * sqrt(fabs(sh_n)));
    return fabs(I) / sqrt(8.0 * tol_n);
}

/* u of vertex i of n: target f(ua) + (i/n)(f(ub) - f(ua)); the approximation's
 * inverse of the target, then two Newton steps on f(u) - target.  Every
 * iterate stays inside [ua, ub]; a step is skipped where f' vanishes. */
double orc_refined_u(double ua, double ub, int64_t i, int64_t n) {
    double lo = fmin(ua, ub), hi = fmax(ua, ub);
    double Fa = orc_f_exact(ua), Fb = orc_f_exact(ub);
    double target = Fa + (Fb - Fa) * ((double)i / (double)n);
    double u = fmin(hi, fmax(lo, orc_f_approx_inv(target)));
    for (int it = 0; it < 2; it++) {
        double d = orc_f_exact_deriv(u);
        if (d > 0.0) u = fmin(hi, fmax(lo, u - (orc_f_exact(u) - target) / d));
    }
    return u;
}

static double line_s_refined(const ES* e, double sh_n, double a, double b, int64_t i, int64_t n) {
    if (i == 0) return a;
    if (i == n) return b;
    double ua = -1.0 - 2.0 * sh_n * es_kn(e, a), ub = -1.0 - 2.0 * sh_n * es_kn(e, b);
    double fr = (double)i / (double)n;
    if (!fx_diff_resolved(ua, ub)) return a + (b - a) * fr;
    double ui = orc_refined_u(ua, ub, i, n);
    return a + (b - a) * ((ui - ua) / (ub - ua));
}

/* Fill flattening (offset 0; Algorithm 1 flattens the source curve itself):
 * the line density of Section 2.1 is sqrt|kappa|, so on the unit ES, whose
 * normalised curvature kappa_n(s) = k0 + k1 (s - 1/2) is linear,
 *   N = int_a^b sqrt|kappa_n| ds / sqrt(8 tol_n),   tol_n = tol / L,
 * and int sqrt|kappa_n| ds = (G(kappa_b) - G(kappa_a)) / k1 with
 * G(k) = (2/3) k |k|^(1/2) -- the 2/3-power law of Section 2.2.  When the
 * curvature hardly changes over the range, the integrand is constant. */
static double fill_G(double k) { return (2.0 / 3.0) * k * sqrt(fabs(k)); }

double orc_fill_count(double k0, double k1, double a, double b, double tol_n) {
    double ka = k0 + k1 * (a - 0.5), kb = k0 + k1 * (b - 0.5);
    double I;
    if (fabs(kb - ka) <= 1e-9 * fmax(fabs(ka), fabs(kb)) || k1 == 0.0)
        I = sqrt(fabs(0.5 * (ka + kb))) * (b - a);
    else
        I = (fill_G(kb) - fill_G(ka)) / k1;
    return fabs(I) / sqrt(8.0 * tol_n);
}

/* parameter of vertex i of n: equal steps of G between kappa_n(a) and kappa_n(b) */
static double fill_s(const ES* e, double a, double b, int64_t i, int64_t n) {
    if (i == 0) return a;
    if (i == n) return b;
    double fr = (double)i / (double)n;
    double ka = es_kn(e, a), kb = es_kn(e, b);
    if (fabs(kb - ka) <= 1e-9 * fmax(fabs(ka), fabs(kb)) || e->k1 == 0.0) return a + (b - a) * fr;
    double Gi = fill_G(ka) + (fill_G(kb) - fill_G(ka)) * fr;
    /* invert G: k = sign(G) (3|G|/2)^(2/3) */
    double ki = copysign(pow(1.5 * fabs(Gi), 2.0 / 3.0), Gi);
    double si = a + (ki - ka) / e->k1;
    return fmin(b, fmax(a, si));
}

/* Section 5: arcs for the ES parallel curve over a range of arc length S,
 * curvature slope kp (per unit length^2), half-width h. */
double orc_arc_count(double S, double kp, double h, double tol) {
    return S * cbrt(fabs(kp) * (1.0 + 0.4 * fabs(h * S * kp)) / (120.0 * tol));
}

/* Section 6: evolute lines over [a, b] of the unit ES.  The evolute's
 * density is |s - s_infl|^(-1/2) in arc length of the ES, so the count is
 * 2 |sqrt|b - s_infl| - sqrt|a - s_infl|| scaled to physical length. */
double orc_evolute_count(double k0, double k1, double L, double a, double b, double tol) {
    if (k1 == 0.0) return 0.0;
    double s0 = 0.5 - k0 / k1;
    double ga = sqrt(fabs(a - s0)), gb = sqrt(fabs(b - s0));
    return 2.0 * sqrt(L) * (b - a) / (ga + gb) / sqrt(8.0 * tol);
}

static double evolute_s(const ES* e, double a, double b, int64_t i, int64_t n) {
    if (i == 0) return a;
    if (i == n) return b;
    double fr = (double)i / (double)n;
    if (e->k1 == 0.0) return a + (b - a) * fr;
    double s0 = 0.5 - e->k0 / e->k1;
    double ga = sqrt(fabs(a - s0)), gb = sqrt(fabs(b - s0));
    double gi = ga + fr * (gb - ga);
    return a + (b - a) * fr * (gi + ga) / (ga + gb);
}

/* Section 2.1: exact arc metric for a circular arc of radius r turning by
 * angle ang: n = ang / (2 acos(1 - tol / r)). */
static int64_t round_count(Em* em, double ang, double r) {
    double x = 1.0 - em->cfg->tol_flat / r;
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    double step = 2.0 * acos(x);
    return count_of(em, ang / step);
}

/* Menger curvature of the circle through a, m, b, signed for a -> b */
static double menger(V2 a, V2 m, V2 b) {
    double cr = vcross(vsub(m, a), vsub(b, m));
    double d = vlen(vsub(m, a)) * vlen(vsub(b, m)) * vlen(vsub(b, a));
    return d > 0.0 ? 2.0 * cr / d : 0.0;
}

/* ------------------------------------------------------------------ */
/* Emission of one ES piece on one side                                */
/* ------------------------------------------------------------------ */
static int64_t offset_n(Em* em, const ES* e, double sh, double a, double b) {
    const Cfg* cfg = em->cfg;
    if (cfg->arcs) {
        double S = (b - a) * e->L;
        double kp = e->k1 / (e->L * e->L);
        /* k1 grows with th1 - th0, a difference of two FP32 angles: its relative
         * FP32 error, and 2/3 of it in the cube-root count, is amplified by
         * (|th0| + |th1|) / |th1 - th0| */
        double saved = em->cond;
        double dlt = fabs(e->th1 - e->th0);
        double ck = dlt > 0.0 ? (2.0 * saved + EPS32 * (fabs(e->th0) + fabs(e->th1))) / dlt * (2.0 / 3.0) : 0.0;
        if (ck > em->cond) em->cond = ck;
        int64_t n = count_of(em, orc_arc_count(S, kp, fabs(sh), cfg->tol_flat));
        em->cond = saved;
        return n;
    }
    if (sh == 0.0) return count_of(em, orc_fill_count(e->k0, e->k1, a, b, cfg->tol_flat / e->L));
    if (cfg->refine) return count_of(em, orc_line_count_exact(e->k0, e->k1, sh / e->L, a, b, cfg->tol_flat / e->L));
    return count_of(em, orc_line_count(e->k0, e->k1, sh / e->L, a, b, cfg->tol_flat / e->L));
}

static double offset_sample(const ES* e, double sh, int arcs, int refine, double a, double b, int64_t i,
                            int64_t n) {
    if (arcs) {
        if (i == 0) return a;
        if (i == n) return b;
        return a + (b - a) * ((double)i / (double)n);
    }
    if (sh == 0.0) return fill_s(e, a, b, i, n);
    if (refine) return line_s_refined(e, sh / e->L, a, b, i, n);
    return line_s(e, sh / e->L, a, b, i, n);
}

/* forward offset on [a, b]; reverse != 0 emits it backwards */
static void offset_range(Em* em, const ES* e, double sh, double a, double b, int reverse, int64_t n) {
    int arcs = em->cfg->arcs;
    V2 prev = es_offset(e, a, sh);
    double sprev = a;
    V2* pts = malloc(sizeof(V2) * (size_t)(n + 1));
    double* ks = malloc(sizeof(double) * (size_t)(n + 1));
    pts[0] = prev;
    for (int64_t i = 1; i <= n; i++) {
        double s = offset_sample(e, sh, arcs, em->cfg->refine, a, b, i, n);
        V2 cur = es_offset(e, s, sh);
        ks[i - 1] = arcs ? menger(prev, es_offset(e, 0.5 * (sprev + s), sh), cur) : 0.0;
        pts[i] = cur;
        prev = cur;
        sprev = s;
    }
    if (!reverse) {
        for (int64_t i = 0; i < n; i++) emit(em, pts[i], pts[i + 1], ks[i], PK_OFFSET);
    } else {
        for (int64_t i = n - 1; i >= 0; i--) emit(em, pts[i + 1], pts[i], -ks[i], PK_OFFSET_REV);
    }
    free(pts);
    free(ks);
}

/* Section 6 / Algorithm 2: where the offset runs backwards (w < 0) emit the
 * path offset(a) -> evolute(a .. b) -> offset(b) twice, then the offset
 * itself reversed, so every vertex stays balanced and windings stay >= 0. */
static void evolute_patch(Em* em, const ES* e, double sh, double a, double b) {
    const Cfg* cfg = em->cfg;
    int64_t n_o = offset_n(em, e, sh, a, b);
    int64_t n_e = count_of(em, orc_evolute_count(e->k0, e->k1, e->L, a, b, cfg->tol_flat));
    V2 oa = es_offset(e, a, sh), ob = es_offset(e, b, sh);
    V2* ev = malloc(sizeof(V2) * (size_t)(n_e + 1));
    for (int64_t i = 0; i <= n_e; i++) ev[i] = es_evolute(e, evolute_s(e, a, b, i, n_e));
    for (int rep = 0; rep < 2; rep++) {
        emit(em, oa, ev[0], 0.0, PK_CONNECT);
        for (int64_t i = 0; i < n_e; i++) emit(em, ev[i], ev[i + 1], 0.0, PK_EVOLUTE);
        emit(em, ev[n_e], ob, 0.0, PK_CONNECT);
    }
    free(ev);
    offset_range(em, e, sh, a, b, 1, n_o);
}

/* primitives piece_side emits for one side (counts only) */
static int64_t side_count(Em* em, const ES* e, int sigma, double h) {
    double sh = sigma * h;
    if (e->degenerate) return 1;
    double sh_n = sh / e->L;
    double w0 = 1.0 + sh_n * es_kn(e, 0.0), w1 = 1.0 + sh_n * es_kn(e, 1.0);
    double ts = (w0 * w1 >= 0.0) ? 1.0 : w0 / (w0 - w1);
    int64_t n = 0;
    double ea = 0.0, eb = 0.0, oa = 0.0, ob = ts;
    int has_evo = 0;
    if (w0 >= 0.0) {
        if (ts < 1.0) { has_evo = 1; ea = ts; eb = 1.0; }
    } else {
        has_evo = 1; ea = 0.0; eb = ts; oa = ts; ob = 1.0;
        if (!(ts < 1.0)) oa = ob = -1.0;
    }
    if (oa >= 0.0) n += offset_n(em, e, sh, oa, ob);
    if (has_evo)
        n += offset_n(em, e, sh, ea, eb) + 2 * (count_of(em, orc_evolute_count(e->k0, e->k1, e->L, ea, eb, em->cfg->tol_flat)) + 2);
    return n;
}

/* A piece's counts are functions of its fit angles, which FP32 resolves only to
 * about em->cond: when moving the angles by that much changes the piece's
 * primitive count, the count is not determined in FP32 and the segment is
 * fragile.  (Near-straight pieces whose control points are large compared with
 * their size, such as short dash parts far from the origin, are the typical case.) */
static void check_count_sensitivity(Em* em, const ES* e, double h) {
    double d = em->cond;
    if (e->degenerate || !(d > 0.0) || !isfinite(d)) return;
    orc_result scratch;
    memset(&scratch, 0, sizeof scratch);
    Em q = *em;
    q.r = &scratch;
    int64_t base = side_count(&q, e, +1, h) + (h != 0.0 ? side_count(&q, e, -1, h) : 0);
    for (int k = 0; k < 4; k++) {
        ES e2 = *e;
        e2.th0 += (k & 1) ? d : -d;
        e2.th1 += (k & 2) ? d : -d;
        es_setup(&e2);
        int64_t n2 = side_count(&q, &e2, +1, h) + (h != 0.0 ? side_count(&q, &e2, -1, h) : 0);
        if (n2 != base) {
            em->sens = 1;
            em->margin = 0.0;
            return;
        }
    }
}

static void piece_side(Em* em, const ES* e, int sigma, double h) {
    em->flip = sigma < 0;
    em->side = sigma;
    double sh = sigma * h;
    if (e->degenerate) {
        emit(em, shared_offset(e->p0, e->q0, sh), shared_offset(e->p1, e->q1, sh), 0.0, PK_DEGEN);
        return;
    }
    double sh_n = sh / e->L;
    double x0 = sh_n * es_kn(e, 0.0), x1 = sh_n * es_kn(e, 1.0);
    double w0 = 1.0 + x0, w1 = 1.0 + x1;
    upd(em, fabs(w0) / fmax(1.0, fabs(x0)));
    upd(em, fabs(w1) / fmax(1.0, fabs(x1)));
    double ts = (w0 * w1 >= 0.0) ? 1.0 : w0 / (w0 - w1);
    if (w0 >= 0.0) {
        offset_range(em, e, sh, 0.0, ts, 0, offset_n(em, e, sh, 0.0, ts));
        if (ts < 1.0) evolute_patch(em, e, sh, ts, 1.0);
    } else {
        evolute_patch(em, e, sh, 0.0, ts);
        if (ts < 1.0) offset_range(em, e, sh, ts, 1.0, 0, offset_n(em, e, sh, ts, 1.0));
    }
}

/* ------------------------------------------------------------------ */
/* Segments                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int is_line;
    V2 p[4];
    /* 0 for a segment read from the input; for a part cut out by dashing, the
     * magnitude at which its computed control points are rounded to FP32 */
    double abs_mag;
} Seg;

static V2 cubic_eval(const Seg* s, double t) {
    double mt = 1.0 - t;
    double b0 = mt * mt * mt, b1 = 3.0 * mt * mt * t, b2 = 3.0 * mt * t * t, b3 = t * t * t;
    return vec(b0 * s->p[0].x + b1 * s->p[1].x + b2 * s->p[2].x + b3 * s->p[3].x,
               b0 * s->p[0].y + b1 * s->p[1].y + b2 * s->p[2].y + b3 * s->p[3].y);
}

static V2 cubic_deriv(const Seg* s, double t) {
    double mt = 1.0 - t;
    V2 d01 = vsub(s->p[1], s->p[0]), d12 = vsub(s->p[2], s->p[1]), d23 = vsub(s->p[3], s->p[2]);
    return vmul(vadd(vadd(vmul(d01, mt * mt), vmul(d12, 2.0 * mt * t)), vmul(d23, t * t)), 3.0);
}

/* Section 7.3: a (near-)zero derivative is re-sampled at a parameter moved
 * by deriv_dt toward the inside of the piece that ends (or, at t = 0,
 * starts) there. */
static V2 deriv_robust(Em* em, const Seg* s, double t) {
    if (s->is_line) return vsub(s->p[3], s->p[0]);
    V2 d = cubic_deriv(s, t);
    double S = vlen(vsub(s->p[1], s->p[0])) + vlen(vsub(s->p[2], s->p[1])) + vlen(vsub(s->p[3], s->p[2]));
    double thr = em->cfg->deriv_eps * S;
    double m = vlen(d);
    double saved = em->cond;
    /* |B'| is a weighted sum of control-point differences: FP32 error ~4 eps32 S */
    em->cond = EPS32 * 4.0 / em->cfg->deriv_eps;
    if (thr > 0.0) upd(em, fabs(m - thr) / thr);
    em->cond = saved;
    if (m < thr) {
        double tt = t > 0.0 ? t - em->cfg->deriv_dt : t + em->cfg->deriv_dt;
        d = cubic_deriv(s, tt);
        if (d.x == 0.0 && d.y == 0.0) d = vsub(s->p[3], s->p[0]);
        if (d.x == 0.0 && d.y == 0.0) d = vec(1.0, 0.0);
    }
    return d;
}

static V2 start_tangent(Em* em, const Seg* s) { return deriv_robust(em, s, 0.0); }

/* largest control-point offset from the segment start (the scale of FP32 rounding
 * in the translation-invariant evaluation) */
static double seg_scale(const Seg* s) {
    double m = 0.0;
    for (int k = 1; k < 4; k++) m = fmax(m, fmax(fabs(s->p[k].x - s->p[0].x), fabs(s->p[k].y - s->p[0].y)));
    return fmax(m, s->abs_mag);
}

/* Algorithm 2: adaptive cubic -> ES subdivision with the (t0_u, dt) stack.
 * Each accepted piece is emitted on side +h then side -h.  Returns the
 * derivative sampled at t = 1 (the end tangent). */
static V2 stroke_pieces(Em* em, const Seg* s, double h, int64_t seg_index) {
    orc_result* r = em->r;
    const Cfg* cfg = em->cfg;
    uint32_t t0_u = 0;
    double dt = 1.0;
    int depth = 0;
    V2 p0 = s->p[0];
    V2 q0 = deriv_robust(em, s, 0.0);
    V2 q_end = q0;
    for (;;) {
        double t0 = (double)t0_u * dt;
        if (t0 >= 1.0) break;
        double t1 = t0 + dt;
        V2 p1 = (t1 == 1.0) ? s->p[3] : cubic_eval(s, t1);
        V2 q1 = s->is_line ? q0 : deriv_robust(em, s, t1);
        double pp0[2] = {p0.x, p0.y}, pp1[2] = {p1.x, p1.y}, qq0[2] = {q0.x, q0.y}, qq1[2] = {q1.x, q1.y};
        double fit[4];
        orc_fit(pp0, pp1, qq0, qq1, dt, fit);
        r->n_fit++;
        /* in FP32 the chord is a difference of points evaluated relative to the
         * segment start: its direction, and every angle and count derived from
         * it, carries about 4 eps32 * (size of the control polygon) / chord */
        /* ... and the tangent angles carry eps32 * (polygon size) / |q| too,
         * which dominates near a (near-)cusp where the derivative is small */
        em->cond = fit[2] > 0.0 ? EPS32 * 4.0 * seg_scale(s) * (1.0 / fit[2] + 3.0 / vlen(q0) + 3.0 / vlen(q1))
                                : INFINITY;
        double err = fit[3];
        double tol = cfg->tol_fit;
        int ok = err <= tol;
        ES e;
        memset(&e, 0, sizeof e);
        e.p0 = p0; e.p1 = p1; e.q0 = q0; e.q1 = q1;
        e.th0 = fit[0]; e.th1 = fit[1]; e.chord_len = fit[2];
        e.t0 = t0; e.t1 = t1;
        if (ok && fit[2] > 0.0) {
            /* pieces outside the range where the Appendix A polynomials hold
             * (chord/arc ratio below C_MIN) are subdivided further */
            double k1, c;
            orc_gh(e.th0 + e.th1, e.th1 - e.th0, &k1, &c);
            upd(em, fabs(c - C_MIN) / C_MIN);
            if (c < C_MIN) ok = 0;
        }
        if (!ok && depth < cfg->max_depth) {
            if (isfinite(err)) upd(em, fabs(err - tol) / tol);
            t0_u *= 2u;
            dt *= 0.5;
            depth++;
            continue;
        }
        if (ok) upd(em, fabs(err - tol) / tol);
        if (fit[2] == 0.0) e.degenerate = 1;
        else es_setup(&e);
        int32_t pid = push_piece(r, &e, seg_index, em->cond);
        em->piece = pid;
        r->seg_npiece[r->n_seg - 1]++;
        piece_side(em, &e, +1, h);
        if (h != 0.0) piece_side(em, &e, -1, h);   /* a fill (h = 0) has one forward side */
        check_count_sensitivity(em, &e, h);
        em->piece = -1;
        em->cond = 0.0;
        /* pop the stack */
        t0_u += 1u;
        int shift = 0;
        while (((t0_u >> shift) & 1u) == 0u && shift < 31) shift++;
        t0_u >>= shift;
        dt *= (double)(1u << shift);
        depth -= shift;
        p0 = p1;
        q0 = q1;
        q_end = q1;
    }
    return q_end;
}

/* ------------------------------------------------------------------ */
/* Joins and caps (SVG semantics)                                      */
/* ------------------------------------------------------------------ */
enum { J_BEVEL = 0, J_MITER = 1, J_ROUND = 2 };
enum { C_BUTT = 0, C_SQUARE = 1, C_ROUND = 2 };

/* polyline of a circular arc about P from A by signed angle ang (n steps), ending exactly at B */
static void round_poly(Em* em, V2 P, V2 A, V2 B, double ang, int64_t n, int kind) {
    V2 prev = A;
    V2 ra = vsub(A, P);
    for (int64_t i = 1; i <= n; i++) {
        V2 cur = (i == n) ? B : vadd(P, vrot(ra, ang * (double)i / (double)n));
        emit(em, prev, cur, 0.0, kind);
        prev = cur;
    }
}

static void join(Em* em, V2 P, V2 Ti, V2 To, double h, int style, double ml, double si, double so) {
    V2 AR = shared_offset(P, Ti, h), BR = shared_offset(P, To, h);
    V2 AL = shared_offset(P, Ti, -h), BL = shared_offset(P, To, -h);
    double cr = vcross(Ti, To), dp = vdot(Ti, To);
    double li = vlen(Ti), lo = vlen(To);
    /* tangents are sums of control-point differences (scales si, so) */
    em->cond = EPS32 * 4.0 * fmax(si / li, so / lo);
    upd(em, fabs(cr) / (li * lo));
    int left = cr >= 0.0;
    double alpha = atan2(fabs(cr), dp);
    int sig_out = left ? +1 : -1;
    for (int pass = 0; pass < 2; pass++) {
        int sigma = pass == 0 ? +1 : -1;
        em->flip = sigma < 0;
        em->side = sigma;
        V2 A = sigma > 0 ? AR : AL, B = sigma > 0 ? BR : BL;
        if (sigma != sig_out) {               /* inner contour through the joint */
            emit(em, A, P, 0.0, PK_JOIN_INNER);
            emit(em, P, B, 0.0, PK_JOIN_INNER);
            continue;
        }
        if (style == J_MITER) {
            double cosa = dp / (li * lo);
            double q = (1.0 + cosa) * ml * ml * 0.5;
            upd(em, fabs(q - 1.0));
            if (q >= 1.0) {
                double sc = sigma * h / (1.0 + cosa);
                V2 Ri = vec(Ti.y / li, -Ti.x / li), Ro = vec(To.y / lo, -To.x / lo);
                V2 M = vec(P.x + sc * (Ri.x + Ro.x), P.y + sc * (Ri.y + Ro.y));
                emit(em, A, M, 0.0, PK_JOIN_OUTER);
                emit(em, M, B, 0.0, PK_JOIN_OUTER);
            } else {
                emit(em, A, B, 0.0, PK_JOIN_OUTER);
            }
        } else if (style == J_ROUND) {
            if (em->cfg->arcs) {
                emit(em, A, B, sigma / h, PK_JOIN_OUTER);
            } else {
                int64_t n = round_count(em, alpha, h);
                round_poly(em, P, A, B, sigma * alpha, n, PK_JOIN_OUTER);
            }
        } else {
            emit(em, A, B, 0.0, PK_JOIN_OUTER);
        }
    }
    em->cond = 0.0;
}

/* end cap: from the +h side to the -h side, bulging along T */
static void end_cap(Em* em, V2 P, V2 T, double h, int cap) {
    V2 AR = shared_offset(P, T, h), AL = shared_offset(P, T, -h);
    em->flip = 0;
    em->side = 0;
    if (cap == C_BUTT) {
        emit(em, AR, AL, 0.0, PK_CAP);
    } else if (cap == C_SQUARE) {
        double l = vlen(T);
        V2 E = vec(h * T.x / l, h * T.y / l);
        V2 a = vadd(AR, E), b = vadd(AL, E);
        emit(em, AR, a, 0.0, PK_CAP);
        emit(em, a, b, 0.0, PK_CAP);
        emit(em, b, AL, 0.0, PK_CAP);
    } else {
        if (em->cfg->arcs) emit(em, AR, AL, 1.0 / h, PK_CAP);
        else round_poly(em, P, AR, AL, ORC_PI, round_count(em, ORC_PI, h), PK_CAP);
    }
}

/* start cap: from the -h side to the +h side, bulging against T */
static void start_cap(Em* em, V2 P, V2 T, double h, int cap) {
    V2 BR = shared_offset(P, T, h), BL = shared_offset(P, T, -h);
    em->flip = 0;
    em->side = 0;
    if (cap == C_BUTT) {
        emit(em, BL, BR, 0.0, PK_CAP);
    } else if (cap == C_SQUARE) {
        double l = vlen(T);
        V2 E = vec(-h * T.x / l, -h * T.y / l);
        V2 a = vadd(BL, E), b = vadd(BR, E);
        emit(em, BL, a, 0.0, PK_CAP);
        emit(em, a, b, 0.0, PK_CAP);
        emit(em, b, BR, 0.0, PK_CAP);
    } else {
        if (em->cfg->arcs) emit(em, BL, BR, 1.0 / h, PK_CAP);
        else round_poly(em, P, BL, BR, ORC_PI, round_count(em, ORC_PI, h), PK_CAP);
    }
}

/* ------------------------------------------------------------------ */
/* Subpaths, dashing, paths                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    Seg* seg;
    int64_t n, cap;
    int closed;
    int drawn;        /* any drawing verb after the moveto */
    V2 start;
} Sub;

static void sub_push(Sub* sp, Seg s) {
    if (sp->n == sp->cap) {
        sp->cap = sp->cap ? 2 * sp->cap : 16;
        sp->seg = realloc(sp->seg, sizeof(Seg) * (size_t)sp->cap);
    }
    sp->seg[sp->n++] = s;
}

typedef struct {
    double h, ml;
    int join, cap;
    int fill;           /* 1: a filled path (Algorithm 1: the source curve, offset 0) */
    int has_xf;         /* the path's affine transform (Section 8.2) is not the identity */
    double xf[6];       /* x' = a x + c y + e, y' = b x + d y + f for (a b c d e f) */
} Style;

/* Section 8.2 gives every path an affine transform.  The outline is that of
 * the transformed path: control points map exactly (an affine image of a Bezier
 * is the Bezier of the images), dashes are measured before the transform, and
 * the half-width is scaled by sqrt|det| of the linear part, which is the
 * transformed stroke for a similarity and an isotropic pen otherwise. */
static V2 xf_apply(const double* m, V2 p) { return vec(m[0] * p.x + m[2] * p.y + m[4], m[1] * p.x + m[3] * p.y + m[5]); }

static double xf_scale(const double* m) { return sqrt(fabs(m[0] * m[3] - m[1] * m[2])); }

static Sub xf_sub(const Sub* sp, const double* m) {
    Sub t = *sp;
    t.seg = malloc(sizeof(Seg) * (size_t)(sp->n ? sp->n : 1));
    t.cap = sp->n;
    double sc = xf_scale(m);
    for (int64_t j = 0; j < sp->n; j++) {
        Seg g = sp->seg[j];
        /* the transformed control points are computed, so FP32 rounds them at
         * the magnitude of the terms of the transform */
        double mag = 0.0;
        for (int k = 0; k < 4; k++) {
            V2 q = g.p[k];
            mag = fmax(mag, fmax(fabs(m[0] * q.x) + fabs(m[2] * q.y) + fabs(m[4]),
                                 fabs(m[1] * q.x) + fabs(m[3] * q.y) + fabs(m[5])));
            g.p[k] = xf_apply(m, q);
        }
        g.abs_mag = fmax(g.abs_mag * sc, 2.0 * mag);
        t.seg[j] = g;
    }
    t.start = xf_apply(m, sp->start);
    return t;
}

/* fill one decoded subpath (Algorithm 1, fill branch): each segment, the
 * closing line included, flattened at offset 0 in its own direction; the
 * cap marker outputs nothing */
static void fill_sub(Em* em, const Sub* sp, int path) {
    orc_result* r = em->r;
    for (int64_t j = 0; j < sp->n; j++) {
        const Seg* s = &sp->seg[j];
        res_push_seg(r, s->is_line == 2 ? 1 : 0, path);
        int64_t si = r->n_seg - 1;
        em->margin = INFINITY;
        em->raw_margin = INFINITY;
        em->sens = 0;
        em->piece = -1;
        Seg sl = *s;
        if (sl.is_line == 2) sl.is_line = 1;
        stroke_pieces(em, &sl, 0.0, si);
        em->piece = -1;
        r->seg_count[si] = r->n_prim - r->seg_first_prim[si];
        r->seg_margin[si] = em->margin;
        r->seg_raw_margin[si] = em->raw_margin;
        r->seg_sens[si] = (int8_t)em->sens;
    }
    res_push_seg(r, 2, path);
    r->seg_margin[r->n_seg - 1] = INFINITY;
}

/* stroke one decoded subpath: its segments, then the cap marker */
static void stroke_sub(Em* em, const Sub* sp, const Style* st, int path) {
    orc_result* r = em->r;
    int64_t n = sp->n;
    if (n == 0) {
        res_push_seg(r, 2, path);
        em->margin = INFINITY;
        em->raw_margin = INFINITY;
        em->sens = 0;
        if (st->cap != C_BUTT) {
            end_cap(em, sp->start, vec(1.0, 0.0), st->h, st->cap);
            start_cap(em, sp->start, vec(1.0, 0.0), st->h, st->cap);
        }
        r->seg_count[r->n_seg - 1] = r->n_prim - r->seg_first_prim[r->n_seg - 1];
        r->seg_margin[r->n_seg - 1] = em->margin;
        r->seg_raw_margin[r->n_seg - 1] = em->raw_margin;
        r->seg_sens[r->n_seg - 1] = (int8_t)em->sens;
        return;
    }
    for (int64_t j = 0; j < n; j++) {
        const Seg* s = &sp->seg[j];
        int is_close = sp->closed && j == n - 1 && s->is_line == 2;
        res_push_seg(r, is_close ? 1 : 0, path);
        int64_t si = r->n_seg - 1;
        em->margin = INFINITY;
        em->raw_margin = INFINITY;
        em->sens = 0;
        em->piece = -1;
        Seg sl = *s;
        if (sl.is_line == 2) sl.is_line = 1;
        V2 Tend = stroke_pieces(em, &sl, st->h, si);
        em->piece = -1;
        V2 P = sl.p[3];
        if (j + 1 < n || sp->closed) {
            Seg nx = sp->seg[j + 1 < n ? j + 1 : 0];
            if (nx.is_line == 2) nx.is_line = 1;
            V2 To = start_tangent(em, &nx);
            join(em, P, Tend, To, st->h, st->join, st->ml, 3.0 * seg_scale(&sl), 3.0 * seg_scale(&nx));
        } else {
            /* the cap's direction is the sampled tangent: like a join's, a sum of
             * control-point differences resolved to FP32 at the segment's scale */
            em->pcond = EPS32 * 4.0 * 3.0 * seg_scale(&sl) / vlen(Tend);
            end_cap(em, P, Tend, st->h, st->cap);
            em->pcond = -1.0;
        }
        r->seg_count[si] = r->n_prim - r->seg_first_prim[si];
        r->seg_margin[si] = em->margin;
        r->seg_raw_margin[si] = em->raw_margin;
        r->seg_sens[si] = (int8_t)em->sens;
    }
    /* cap marker: start cap of an open subpath */
    res_push_seg(r, 2, path);
    int64_t mi = r->n_seg - 1;
    em->margin = INFINITY;
    em->raw_margin = INFINITY;
    em->sens = 0;
    if (!sp->closed) {
        Seg f = sp->seg[0];
        if (f.is_line == 2) f.is_line = 1;
        V2 T0 = start_tangent(em, &f);
        em->pcond = EPS32 * 4.0 * 3.0 * seg_scale(&f) / vlen(T0);
        start_cap(em, f.p[0], T0, st->h, st->cap);
        em->pcond = -1.0;
    }
    r->seg_count[mi] = r->n_prim - r->seg_first_prim[mi];
    r->seg_margin[mi] = em->margin;
    r->seg_raw_margin[mi] = em->raw_margin;
    r->seg_sens[mi] = (int8_t)em->sens;
}

/* 16-point Gauss-Legendre value of int_a^b |B'(t)| dt */
static double speed_gl(const Seg* s, double a, double b) {
    double acc = 0.0;
    for (int i = 0; i < GL_N; i++) acc += gl_w[i] * vlen(cubic_deriv(s, a + 0.5 * (b - a) * (gl_x[i] + 1.0)));
    return 0.5 * (b - a) * acc;
}

/* adaptive bisection: accept [a, b] when its two halves agree with the whole */
static double speed_adapt(const Seg* s, double a, double b, double whole, double eps, int depth) {
    double m = 0.5 * (a + b);
    double l = speed_gl(s, a, m), r = speed_gl(s, m, b);
    if (depth >= 40 || fabs(l + r - whole) <= eps) return l + r;
    return speed_adapt(s, a, m, l, 0.5 * eps, depth + 1) + speed_adapt(s, m, b, r, 0.5 * eps, depth + 1);
}

/* FP64 arc length of a segment over [0, t]: adaptive Gauss-Legendre on |B'|
 * to ~1e-14 of the control polygon's length (a near-cusp |B'| has a sharp
 * minimum that fixed panels resolve only to ~1e-5) */
static double seg_len(const Seg* s, double t) {
    if (s->is_line) return vlen(vsub(s->p[3], s->p[0])) * t;
    if (t <= 0.0) return 0.0;
    double poly = vlen(vsub(s->p[1], s->p[0])) + vlen(vsub(s->p[2], s->p[1])) + vlen(vsub(s->p[3], s->p[2]));
    return speed_adapt(s, 0.0, t, speed_gl(s, 0.0, t), 1e-14 * poly, 0);
}

/* parameter at which the arc length reaches target (bisection) */
static double seg_param_at(const Seg* s, double target, double total) {
    if (s->is_line) return total > 0.0 ? target / total : 0.0;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 80; it++) {
        double mid = 0.5 * (lo + hi);
        if (seg_len(s, mid) < target) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* the part of a segment over [ta, tb] (de Casteljau) */
static Seg seg_part(const Seg* s, double ta, double tb) {
    Seg r = *s;
    if (s->is_line) {
        V2 d = vsub(s->p[3], s->p[0]);
        r.p[0] = ta == 0.0 ? s->p[0] : vadd(s->p[0], vmul(d, ta));
        r.p[3] = tb == 1.0 ? s->p[3] : vadd(s->p[0], vmul(d, tb));
        r.p[1] = r.p[0]; r.p[2] = r.p[3];
        double mag = fmax(fmax(fabs(r.p[0].x), fabs(r.p[0].y)), fmax(fabs(r.p[3].x), fabs(r.p[3].y)));
        r.abs_mag = fmax(s->abs_mag, 2.0 * mag);
        return r;
    }
    /* evaluate the sub-cubic's control points via blossoming */
    V2 P[4] = {s->p[0], s->p[1], s->p[2], s->p[3]};
    double u[3];
    for (int k = 0; k < 4; k++) {
        /* blossom arguments: (ta,ta,ta), (ta,ta,tb), (ta,tb,tb), (tb,tb,tb) */
        for (int j = 0; j < 3; j++) u[j] = j < 3 - k ? ta : tb;
        V2 b[4] = {P[0], P[1], P[2], P[3]};
        for (int lvl = 0; lvl < 3; lvl++)
            for (int i = 0; i < 3 - lvl; i++)
                b[i] = vadd(vmul(b[i], 1.0 - u[lvl]), vmul(b[i + 1], u[lvl]));
        r.p[k] = b[0];
    }
    if (ta == 0.0) r.p[0] = s->p[0];
    if (tb == 1.0) r.p[3] = s->p[3];
    /* the dash stream holds these control points in FP32: each carries the
     * rounding (and the few roundings of computing it) at its own magnitude */
    double mag = 0.0;
    for (int k = 0; k < 4; k++) mag = fmax(mag, fmax(fabs(r.p[k].x), fabs(r.p[k].y)));
    r.abs_mag = fmax(s->abs_mag, 2.0 * mag);
    return r;
}

/* Exported for the oracle's own tests: arc length of the segment with control
 * points p[8] (x0 y0 .. x3 y3) over [0, t], and the parameter at arc length target. */
double orc_seg_length(const double* p, int is_line, double t) {
    Seg s;
    s.is_line = is_line;
    s.abs_mag = 0.0;
    for (int k = 0; k < 4; k++) s.p[k] = vec(p[2 * k], p[2 * k + 1]);
    return seg_len(&s, t);
}

double orc_seg_param_at(const double* p, int is_line, double target) {
    Seg s;
    s.is_line = is_line;
    s.abs_mag = 0.0;
    for (int k = 0; k < 4; k++) s.p[k] = vec(p[2 * k], p[2 * k + 1]);
    return seg_param_at(&s, target, seg_len(&s, 1.0));
}

/* SVG dashing: the pattern (repeated twice when its length is odd) starts at
 * dash_offset at the start of every subpath; each "on" interval becomes an
 * open subpath.  Dashes are not merged across the start of a closed subpath. */
static void dash_sub(const Sub* sp, const float* pat, int64_t npat, double offset, Sub** out, int64_t* nout,
                     double* margin) {
    int64_t np = (npat % 2) ? 2 * npat : npat;
    double period = 0.0;
    for (int64_t i = 0; i < np; i++) period += pat[i % npat];
    *out = NULL;
    *nout = 0;
    if (sp->n == 0 || !(period > 0.0)) return;
    /* phase at the start */
    double ph = fmod(offset, period);
    if (ph < 0.0) ph += period;
    int64_t idx = 0;
    while (ph >= pat[idx % npat]) { ph -= pat[idx % npat]; idx = (idx + 1) % np; }
    double left = pat[idx % npat] - ph;     /* length left in the current interval */
    double y_end = 0.0;                     /* arc length from the subpath start */
    int on = (idx % 2) == 0;
    Sub cur;
    memset(&cur, 0, sizeof cur);
    int64_t cap_out = 0;
    if (on) { cur.drawn = 1; cur.start = sp->seg[0].p[0]; }
    for (int64_t j = 0; j < sp->n; j++) {
        Seg s = sp->seg[j];
        if (s.is_line == 2) s.is_line = 1;
        double total = seg_len(&s, 1.0);
        double pos = 0.0;                    /* arc length consumed in this segment */
        double tpos = 0.0;
        while (pos + left < total) {
            double tcut = seg_param_at(&s, pos + left, total);
            if (on && tcut > tpos) sub_push(&cur, seg_part(&s, tpos, tcut));
            if (on) {
                if (*nout == cap_out) { cap_out = cap_out ? 2 * cap_out : 8; *out = realloc(*out, sizeof(Sub) * (size_t)cap_out); }
                (*out)[(*nout)++] = cur;
                memset(&cur, 0, sizeof cur);
            }
            pos += left;
            tpos = tcut;
            idx = (idx + 1) % np;
            left = pat[idx % npat];
            on = !on;
            if (on) { cur.drawn = 1; cur.start = cubic_eval(&s, tcut); if (s.is_line) cur.start = seg_part(&s, tcut, 1.0).p[0]; }
        }
        if (on && tpos < 1.0) sub_push(&cur, tpos == 0.0 ? s : seg_part(&s, tpos, 1.0));
        left -= total - pos;
        /* decision margin: the segment end against the nearest pattern boundary.
         * An FP32 arc length (adaptive quadrature) puts the end within ~2e-7 of
         * the length consumed so far; a boundary within 1e-6 of it can fall on
         * either side.  Reported so that the common fragility threshold 1e-4
         * corresponds to that 1e-6. */
        y_end += total;
        double dist = fmin(left, pat[idx % npat] - left);
        double m = dist / (1e-2 * (y_end + period));
        if (m < *margin) *margin = m;
    }
    if (on) {
        if (*nout == cap_out) { cap_out = cap_out ? 2 * cap_out : 8; *out = realloc(*out, sizeof(Sub) * (size_t)cap_out); }
        (*out)[(*nout)++] = cur;
    } else {
        free(cur.seg);
    }
}

static void finish_sub(Sub* sp) {
    /* Section 8.2: a closed subpath gets a closing line when its end point
     * differs from its start point (marked is_line = 2). */
    if (sp->closed && sp->n > 0) {
        V2 end = sp->seg[sp->n - 1].p[3];
        if (!veq(end, sp->start)) {
            Seg l;
            l.is_line = 2;
            l.abs_mag = 0.0;
            l.p[0] = end; l.p[3] = sp->start; l.p[1] = end; l.p[2] = sp->start;
            sub_push(sp, l);
        }
    }
}

static void handle_sub(Em* em, Sub* sp, const Style* st, int path,
                       const float* dash, int64_t ndash, double dash_offset) {
    if (!sp->drawn) return;
    if (st->fill) {
        /* a filled subpath is closed whether or not it says so (Section 8.2) */
        sp->closed = 1;
        finish_sub(sp);
        if (st->has_xf) {
            Sub t = xf_sub(sp, st->xf);
            fill_sub(em, &t, path);
            free(t.seg);
        } else {
            fill_sub(em, sp, path);
        }
        return;
    }
    finish_sub(sp);
    if (ndash > 0) {
        Sub* parts;
        int64_t np;
        dash_sub(sp, dash, ndash, dash_offset, &parts, &np, &em->dash_margin);
        for (int64_t i = 0; i < np; i++) {
            if (st->has_xf) {
                Sub t = xf_sub(&parts[i], st->xf);
                stroke_sub(em, &t, st, path);
                free(t.seg);
            } else {
                stroke_sub(em, &parts[i], st, path);
            }
            free(parts[i].seg);
        }
        free(parts);
    } else if (st->has_xf) {
        Sub t = xf_sub(sp, st->xf);
        stroke_sub(em, &t, st, path);
        free(t.seg);
    } else {
        stroke_sub(em, sp, st, path);
    }
}

/*
 * Stroke every path of a verb-stream scene.
 *   verbs        MOVE=0 (1 point), LINE=1 (1), CUBIC=2 (3), CLOSE=3 (0), QUAD=4 (2)
 *   pts          2 floats per point
 *   path_verb_off  n_paths + 1 offsets into verbs
 *   styles per path: half width, join (0 bevel 1 miter 2 round),
 *                    cap (0 butt 1 square 2 round), miter limit,
 *                    dash pattern [dash_first, +dash_count) of dash_len, dash offset
 *   fill         per path (may be NULL): nonzero for a filled path -- every subpath
 *                closed, flattened at offset 0, no joins, caps or dashes
 *   xform        per path 6 floats (a b c d e f) or NULL: the path's affine transform
 *   tol, fit_frac, flat_frac: the ES fit uses tol*fit_frac, flattening tol*flat_frac
 *   arcs         0 = lines, 1 = arcs
 * Returns 0, or 2 on malformed input.  Results are appended to *r (zeroed by
 * the caller) and must be released with orc_result_free.
 */
int orc_stroke(const uint8_t* verbs, int64_t n_verbs, const float* pts, int64_t n_pts,
               const uint32_t* path_verb_off, int64_t n_paths,
               const float* hw, const uint8_t* join_style, const uint8_t* cap_style, const float* miter_limit,
               const uint32_t* dash_first, const uint32_t* dash_count, const float* dash_offset,
               const float* dash_len, int64_t n_dash, const uint8_t* fill, const float* xform,
               double tol, double fit_frac, double flat_frac, int arcs, int refine, orc_result* r) {
    Cfg cfg;
    cfg.tol_fit = tol * fit_frac;
    cfg.tol_flat = tol * flat_frac;
    cfg.arcs = arcs;
    cfg.refine = refine && !arcs;
    cfg.max_depth = 16;
    cfg.deriv_eps = 1e-5;
    cfg.deriv_dt = 1.0 / 1024.0;
    cfg.max_count = 65536;
    Em em;
    memset(&em, 0, sizeof em);
    em.r = r;
    em.cfg = &cfg;
    em.piece = -1;
    em.pcond = -1.0;
    int64_t pc = 0;  /* point cursor */
    (void)n_verbs;
    for (int64_t p = 0; p < n_paths; p++) {
        Style st;
        st.h = hw[p]; st.ml = miter_limit[p]; st.join = join_style[p]; st.cap = cap_style[p];
        st.fill = fill ? fill[p] != 0 : 0;
        st.has_xf = 0;
        if (xform) {
            for (int k = 0; k < 6; k++) st.xf[k] = xform[6 * p + k];
            st.has_xf = !(st.xf[0] == 1.0 && st.xf[1] == 0.0 && st.xf[2] == 0.0 && st.xf[3] == 1.0 &&
                          st.xf[4] == 0.0 && st.xf[5] == 0.0);
            if (st.has_xf) st.h *= xf_scale(st.xf);
        }
        const float* dash = dash_count[p] && !st.fill ? dash_len + dash_first[p] : NULL;
        int64_t nd = st.fill ? 0 : dash_count[p];
        if (nd && (int64_t)dash_first[p] + nd > n_dash) return 2;
        int64_t seg_before = r->n_seg;
        em.dash_margin = INFINITY;
        Sub sp;
        memset(&sp, 0, sizeof sp);
        int have = 0;
        V2 cur = vec(0.0, 0.0);
        for (uint32_t vi = path_verb_off[p]; vi < path_verb_off[p + 1]; vi++) {
            int vb = verbs[vi];
            if (vb == 0) {
                if (have) handle_sub(&em, &sp, &st, (int)p, dash, nd, dash_offset[p]);
                sp.n = 0; sp.closed = 0; sp.drawn = 0;
                if (pc + 1 > n_pts) return 2;
                cur = vec(pts[2 * pc], pts[2 * pc + 1]);
                pc += 1;
                sp.start = cur;
                have = 1;
            } else if (vb == 1 || vb == 2 || vb == 4) {
                if (!have) return 2;
                if (sp.closed) {   /* drawing after closepath starts a new subpath at the start point */
                    handle_sub(&em, &sp, &st, (int)p, dash, nd, dash_offset[p]);
                    sp.n = 0; sp.closed = 0; sp.drawn = 0;
                    cur = sp.start;
                }
                Seg s;
                s.p[0] = cur;
                s.abs_mag = 0.0;
                if (vb == 1) {
                    if (pc + 1 > n_pts) return 2;
                    s.is_line = 1;
                    s.p[3] = vec(pts[2 * pc], pts[2 * pc + 1]);
                    s.p[1] = s.p[0]; s.p[2] = s.p[3];
                    pc += 1;
                } else if (vb == 4) {
                    /* a quadratic, degree-elevated to the cubic with the same curve
                     * (all segments become cubics, Section 8.1) */
                    if (pc + 2 > n_pts) return 2;
                    s.is_line = 0;
                    V2 q1 = vec(pts[2 * pc], pts[2 * pc + 1]), q2 = vec(pts[2 * pc + 2], pts[2 * pc + 3]);
                    s.p[1] = vadd(s.p[0], vmul(vsub(q1, s.p[0]), 2.0 / 3.0));
                    s.p[2] = vadd(q2, vmul(vsub(q1, q2), 2.0 / 3.0));
                    s.p[3] = q2;
                    /* the elevated control points are computed, so FP32 rounds them
                     * at the magnitude of the coordinates */
                    s.abs_mag = 2.0 * fmax(fmax(fmax(fabs(s.p[0].x), fabs(s.p[0].y)), fmax(fabs(q1.x), fabs(q1.y))),
                                           fmax(fabs(q2.x), fabs(q2.y)));
                    pc += 2;
                } else {
                    if (pc + 3 > n_pts) return 2;
                    s.is_line = 0;
                    for (int k = 1; k <= 3; k++) s.p[k] = vec(pts[2 * (pc + k - 1)], pts[2 * (pc + k - 1) + 1]);
                    pc += 3;
                }
                sp.drawn = 1;
                /* zero-length segments (every control point at the current point) are dropped */
                if (!(veq(s.p[1], cur) && veq(s.p[2], cur) && veq(s.p[3], cur))) sub_push(&sp, s);
                cur = s.p[3];
            } else if (vb == 3) {
                if (!have) return 2;
                sp.closed = 1;
                sp.drawn = 1;
                cur = sp.start;
            } else {
                return 2;
            }
        }
        if (have) handle_sub(&em, &sp, &st, (int)p, dash, nd, dash_offset[p]);
        free(sp.seg);
        if (r->n_seg == seg_before) {
            res_push_seg(r, 3, (int)p);   /* empty path placeholder */
        }
        for (int64_t k = seg_before; k < r->n_seg; k++) r->seg_dash_margin[k] = em.dash_margin;
    }
    return 0;
}

void orc_result_free(orc_result* r) {
    free(r->seg_kind); free(r->seg_path); free(r->seg_first_prim); free(r->seg_count);
    free(r->seg_margin); free(r->seg_npiece); free(r->seg_dash_margin);
    free(r->seg_raw_margin); free(r->seg_sens);
    free(r->prim); free(r->prim_kind); free(r->prim_side); free(r->prim_piece); free(r->prim_cond);
    free(r->piece); free(r->piece_seg);
    memset(r, 0, sizeof *r);
}
