/*
 * gsr_oracle.c -- FP64 CPU oracle of the 2D-Gaussian surfel sensor renderer.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (arXiv 2503.11731, Sec. III-A "Unified Projection Scheme"):
 *   Eq. 1  P(u,v) = W H (u,v,1)^T, H = [s_u t_u, s_v t_v, mu; 0 0 1]  (4x3)
 *   Eq. 2  [h_u, h_v]^T . P(u,v) = 0 solved for (u,v)
 *   Eq. 3  pinhole planes h_u = (-1,0,0,p_x), h_v = (0,-1,0,p_y)
 *   Eq. 4  cylinder      h_u = (cos phi, 0, -sin phi, 0),
 *                        h_v = (y_n sin phi, -1, y_n cos phi, 0)  (a reading, below)
 *   Eq. 5  LiDAR planes  h_u = (sin az, -cos az, 0, 0),
 *                        h_v = (sin el cos az, sin el sin az, -cos el, 0)
 * and the splatting it cites (3DGS / 2DGS, Sec. II "Scene Representations"):
 * the 2DGS screen-space low-pass fallback and front-to-back alpha compositing.
 * It is a brute-force pass: every pixel (or ray) looks at every surfel, with
 * no tiling, no bounds and no culling beyond the method's own near test.
 *
 * Readings of points the paper leaves open:
 *   - pinhole W = [[fx,0,cx,0],[0,fy,cy,0],[0,0,1,0],[0,0,1,0]] . [R|t], so the
 *     Eq. 3 planes act on pixel-homogeneous coordinates; LiDAR W = [R|t];
 *   - in Eq. 5 the angle inside h_u is the azimuth and the one that appears
 *     alone in h_v is the elevation (the formulas, not the prose, decide);
 *   - Eq. 4 (cylindrical camera): h_v read as the camera-frame plane through
 *     the pixel's ray normal to h_u (see oracle_render_cylindrical);
 *   - an intersection counts only if its depth (camera) or its distance
 *     along the ray (LiDAR) exceeds `near`; surfels whose centre depth
 *     (range) is <= near are culled;
 *   - G3 = exp(-(u^2+v^2)/2) inside u^2+v^2 <= 9; the low-pass term is
 *     exp(-|p-c|^2 / (2 sigma^2)) with sigma^2 = 1/2 (pixels, or LiDAR cells)
 *     inside |p-c| <= 3 sigma; G = max of the valid terms; the contribution
 *     depth is the intersection depth if G3 wins, else the centre depth;
 *   - alpha = min(0.99, o G); alpha < 1/255 is skipped; compositing stops
 *     before a surfel when T (1 - alpha) < 1e-4;
 *   - composite order: centre depth (camera z, LiDAR |mu|, cylinder
 *     horizontal distance) in FP64, ties by index; where two contributing
 *     surfels' depths are closer than an FP32 evaluation of them can
 *     separate, the ray is flagged with the largest change a swap of the
 *     two could make (see or_step), as for every other threshold;
 *   - colour = max(0, sum_lm Y_lm(dir) c_lm + 0.5), real SH with the
 *     Condon-Shortley phase, dir = normalise(mu - sensor origin);
 *   - normal = R's third column, flipped to face the sensor, sensor frame.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ----------------------------------------------------------------------- */
/* Real spherical harmonics from the associated Legendre functions.         */
/* Textbook definition: Y_l^m = sqrt(2) K_l^m cos(m phi) P_l^m(cos theta)    */
/* for m > 0, sqrt(2) K_l^|m| sin(|m| phi) P_l^|m|(cos theta) for m < 0,     */
/* K_l^0 P_l^0 for m = 0, K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), with    */
/* the Condon-Shortley factor (-1)^m inside P_l^m.                           */
/* ----------------------------------------------------------------------- */
static double or_factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

/* P_l^m(x), m >= 0, by the standard three-term recurrence in l. */
static double or_assoc_legendre(int l, int m, double x)
{
    double pmm = 1.0;
    if (m > 0) {
        double s = sqrt((1.0 - x) * (1.0 + x));
        double odd = 1.0;
        for (int i = 1; i <= m; ++i) {
            pmm *= -odd * s; /* (-1)^m (2m-1)!! (1-x^2)^{m/2} */
            odd += 2.0;
        }
    }
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* Y_l^m at the unit direction d. */
double oracle_sh_basis(int l, int m, const double d[3])
{
    int am = m < 0 ? -m : m;
    double ct = d[2];
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double phi = atan2(d[1], d[0]);
    double K = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * or_factorial(l - am) / or_factorial(l + am));
    double P = or_assoc_legendre(l, am, ct);
    if (m == 0) return K * P;
    if (m > 0) return sqrt(2.0) * K * cos(m * phi) * P;
    return sqrt(2.0) * K * sin(am * phi) * P;
}

/* ----------------------------------------------------------------------- */
/* Small linear algebra                                                      */
/* ----------------------------------------------------------------------- */
static void or_cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double or_dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Rotation matrix of the normalised quaternion (w,x,y,z); columns t_u, t_v, n. */
static void or_quat_to_rot(const double q_in[4], double R[3][3])
{
    double nq = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / nq, x = q_in[1] / nq, y = q_in[2] / nq, z = q_in[3] / nq;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* ----------------------------------------------------------------------- */
/* Per-surfel state, independent of the pixel.                               */
/* ----------------------------------------------------------------------- */
typedef struct {
    int culled;        /* centre depth (range) <= near                        */
    double cull_rel;   /* |zc - near| / near: how close the cull decision is  */
    double WH[4][3];   /* Eq. 1: W . H, a 4x3 matrix                         */
    double zc;         /* centre depth (camera z) / centre range (LiDAR |mu|)
                          / horizontal distance (cylinder): the order key     */
    double tau;        /* bound on the error of an FP32 evaluation of zc      */
    int key_exact;     /* not posed, position exactly FP32: key_in holds
                          every operand of the key                           */
    double key_in[3];  /* the centre's coordinates that enter the key with a
                          nonzero coefficient (0 where none does)            */
    double c[2];       /* low-pass centre (pixels, or LiDAR cells)           */
    double c_err[2];   /* bound on the error of an FP32 evaluation of c      */
    double o;          /* opacity, sigmoid of the logit                      */
    double feat[3];    /* camera: colour; LiDAR: intensity, ray drop, 0     */
    double normal[3];  /* sensor frame, facing the sensor                    */
    int n_amb;         /* the facing test n . (mu - origin) is within its FP32
                          error bound of 0: either sign of n is possible     */
    double ms[3];      /* centre in the sensor frame                         */
    double rad;        /* radius of a sphere about the centre that holds the
                          support u^2 + v^2 <= 9 with the near-miss margin    */
    double smin;       /* the smaller scale                                  */
} or_surfel;

typedef struct {
    /* sensor */
    int kind;                        /* 0 pinhole, 1 LiDAR, 2 cylindrical   */
    double Rs[3][3], ts[3];          /* world -> sensor rigid part          */
    double origin[3];                /* sensor origin in world             */
    double fx, fy, cx, cy;           /* cameras                            */
    int width, height;               /* cameras                            */
    int beams, columns;              /* LiDAR                              */
    double el_max, d_el, az0, d_az;  /* radians                            */
    double near_;
    double bg[3];                    /* cameras: the background colour      */
} or_sensor;

static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void or_sensor_from_matrix(or_sensor* S, const double* w2s)
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) S->Rs[i][j] = w2s[i * 4 + j];
        S->ts[i] = w2s[i * 4 + 3];
    }
    /* origin = -R^T t */
    for (int j = 0; j < 3; ++j)
        S->origin[j] = -(S->Rs[0][j] * S->ts[0] + S->Rs[1][j] * S->ts[1] + S->Rs[2][j] * S->ts[2]);
}

/*
 * World-space surfel i after the optional rigid object pose (Sec. III-B,
 * Gaussian inplacing: a model matrix per actor): mu' = R_o mu + t_o,
 * R' = R_o R.  The SH coefficients live in the object frame, so the view
 * direction is rotated back by R_o^T before the basis is evaluated.
 * mag[a] (optional) receives sum_b |R_o[a][b] mu_b| + |t_o[a]|, the size of
 * the terms that make up mu'[a].
 */
static void or_surfel_world(int i, const double* pos, const double* quat, const int* obj_id,
                            const double* obj_pose, double mu[3], double R[3][3], double Ro[3][3],
                            double mag[3])
{
    double Rl[3][3];
    or_quat_to_rot(quat + 4 * i, Rl);
    int k = obj_id ? obj_id[i] : -1;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Ro[a][b] = (a == b) ? 1.0 : 0.0;
    double to[3] = {0, 0, 0};
    if (k >= 0) {
        const double* P = obj_pose + 12 * k;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) Ro[a][b] = P[a * 4 + b];
            to[a] = P[a * 4 + 3];
        }
    }
    for (int a = 0; a < 3; ++a) {
        mu[a] = to[a];
        if (mag) mag[a] = fabs(to[a]);
        for (int b = 0; b < 3; ++b) {
            mu[a] += Ro[a][b] * pos[3 * i + b];
            if (mag) mag[a] += fabs(Ro[a][b] * pos[3 * i + b]);
        }
        for (int b = 0; b < 3; ++b) {
            R[a][b] = 0;
            for (int c = 0; c < 3; ++c) R[a][b] += Ro[a][c] * Rl[c][b];
        }
    }
}

/*
 * Unit roundoff of IEEE single precision, and the error bound of the order
 * key in FP32.  Each sensor-frame component of the centre is a sum of four
 * terms, R_a0 m_0 + R_a1 m_1 + R_a2 m_2 + t_a; evaluated in FP32 (with or
 * without fused multiply-adds, in any order) it is off by at most
 * gamma_4 = 4u / (1 - 4u) times the sum of the terms' magnitudes (the
 * standard bound for inner products, Higham, "Accuracy and Stability of
 * Numerical Algorithms", Sec. 3.1).  A posed object's centre is itself such
 * a sum, whose error the rotation carries on.  The norms of the LiDAR and
 * cylinder keys add at most 3u relative for the squares, the sum and the
 * square root.
 */
#define OR_U32 (1.0 / 16777216.0)
#define OR_GAMMA4 (4.0 * OR_U32 / (1.0 - 4.0 * OR_U32))
/* Roundoffs of the terms' magnitude by which an FP32 evaluation may move
   the surfel plane along its normal or turn the ray: the gamma_4 bound of
   an affine map's four terms, as for the order key. */
#define OR_SOLVE_ROUNDOFF 4.0

/*
 * The FP32 reach of the low-pass centre c (ray units).  An FP32 evaluation
 * places the centre's sensor-frame coordinates within about 4 u |mu_s| (the
 * same estimate as the conditioning of Eq. 2), which turns its direction by
 * that over its distance; an FP32 angle function is within a few ulps of
 * its result (6 u |angle|); and each rounding of the chain that maps the
 * projection to pixels or cells (a quotient, a scale, an offset) costs u
 * times the magnitude it produces.  The bound is capped at one ray spacing.
 */
static void or_centre_error(or_surfel* G, const or_sensor* S)
{
    const double u = OR_U32;
    const double* m = G->ms;
    double ep = OR_SOLVE_ROUNDOFF * u * sqrt(or_dot3(m, m));
    double ex, ey;
    if (S->kind == 0) {
        /* c = f X / Z + c0 */
        double Z = fabs(m[2]) > 1e-30 ? fabs(m[2]) : 1e-30;
        ex = S->fx * ep * (1.0 + fabs(m[0] / Z)) / Z + 3.0 * u * (fabs(G->c[0]) + fabs(S->cx));
        ey = S->fy * ep * (1.0 + fabs(m[1] / Z)) / Z + 3.0 * u * (fabs(G->c[1]) + fabs(S->cy));
    } else if (S->kind == 2) {
        /* c = (c_x + f_x phi, c_y + f_y y / r_h) */
        double rh = G->zc > 1e-30 ? G->zc : 1e-30;
        double phi = atan2(m[0], m[2]);
        ex = S->fx * (ep / rh + 6.0 * u * fabs(phi)) + 3.0 * u * (fabs(G->c[0]) + fabs(S->cx));
        ey = S->fy * ep * (1.0 + fabs(m[1] / rh)) / rh + 3.0 * u * (fabs(G->c[1]) + fabs(S->cy));
    } else {
        /* c = ((az - az0) / d_az - 1/2, (el_max - el) / d_el) */
        double rng = G->zc > 1e-30 ? G->zc : 1e-30;
        double rh = sqrt(m[0] * m[0] + m[1] * m[1]);
        if (rh < 1e-30) rh = 1e-30;
        double az = atan2(m[1], m[0]), el = atan2(m[2], rh);
        ex = (ep / rh + 6.0 * u * fabs(az) + u * (fabs(az) + fabs(S->az0))) / S->d_az + 2.0 * u * (fabs(G->c[0]) + 1.0);
        ey = (ep / rng + 6.0 * u * fabs(el) + u * (fabs(el) + fabs(S->el_max))) / S->d_el + 2.0 * u * (fabs(G->c[1]) + 1.0);
    }
    G->c_err[0] = ex < 1.0 ? ex : 1.0;
    G->c_err[1] = ey < 1.0 ? ey : 1.0;
}

static void or_prepare(or_surfel* G, int i, const or_sensor* S, const double* pos,
                       const double* log_scale, const double* quat, const double* opacity_logit,
                       int sh_degree, const double* sh, const double* intensity,
                       const double* ray_drop, const int* obj_id, const double* obj_pose)
{
    double mu[3], R[3][3], Ro[3][3], mag[3];
    or_surfel_world(i, pos, quat, obj_id, obj_pose, mu, R, Ro, mag);
    double su = exp(log_scale[2 * i + 0]), sv = exp(log_scale[2 * i + 1]);

    /* H (Eq. 1): columns s_u t_u, s_v t_v, mu over a bottom row (0,0,1). */
    double H[4][3];
    for (int a = 0; a < 3; ++a) {
        H[a][0] = su * R[a][0];
        H[a][1] = sv * R[a][1];
        H[a][2] = mu[a];
    }
    H[3][0] = 0; H[3][1] = 0; H[3][2] = 1;

    /* W: pixel-homogeneous view-projection (pinhole) or the rigid transform. */
    double W[4][4];
    double Rt[4][4];
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) Rt[a][b] = S->Rs[a][b];
        Rt[a][3] = S->ts[a];
    }
    Rt[3][0] = Rt[3][1] = Rt[3][2] = 0; Rt[3][3] = 1;
    if (S->kind == 0) {
        double P4[4][4] = {{S->fx, 0, S->cx, 0}, {0, S->fy, S->cy, 0}, {0, 0, 1, 0}, {0, 0, 1, 0}};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                W[a][b] = 0;
                for (int c = 0; c < 4; ++c) W[a][b] += P4[a][c] * Rt[c][b];
            }
    } else {
        memcpy(W, Rt, sizeof(W));
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 3; ++b) {
            G->WH[a][b] = 0;
            for (int c = 0; c < 4; ++c) G->WH[a][b] += W[a][c] * H[c][b];
        }

    /* mu in the sensor frame, and the FP32 error bound of each component */
    int posed = obj_id && obj_id[i] >= 0;
    double ms[3], msmag[3];
    for (int a = 0; a < 3; ++a) {
        ms[a] = S->Rs[a][0] * mu[0] + S->Rs[a][1] * mu[1] + S->Rs[a][2] * mu[2] + S->ts[a];
        double terms = fabs(S->ts[a]), carried = 0.0;
        for (int b = 0; b < 3; ++b) {
            terms += fabs(S->Rs[a][b] * mu[b]);
            carried += fabs(S->Rs[a][b]) * mag[b];
        }
        msmag[a] = OR_GAMMA4 * (terms + (posed ? carried : 0.0));
    }
    for (int a = 0; a < 3; ++a) G->ms[a] = ms[a];
    G->rad = 3.01 * (su > sv ? su : sv);
    G->smin = su < sv ? su : sv;

    /* The key's operands: two unposed surfels whose key computations take
       identical operands get identical FP32 keys in any evaluation order
       (terms with a zero coefficient contribute exact zeros), so an FP32
       sort breaks their tie by index exactly as the FP64 order does. */
    /* (only for positions that are exactly FP32 values, as a table given to
       both sides is: a position the oracle derived in FP64, e.g. by its own
       decode, need not equal the renderer's FP32 one) */
    G->key_exact = !posed;
    for (int b = 0; b < 3; ++b) G->key_exact &= (double)(float)pos[3 * i + b] == pos[3 * i + b];
    for (int b = 0; b < 3; ++b) {
        int used = 0;
        for (int a = 0; a < 3; ++a)
            if ((S->kind == 0 && a == 2) || (S->kind == 2 && a != 1) || S->kind == 1) used |= S->Rs[a][b] != 0.0;
        G->key_in[b] = used ? pos[3 * i + b] : 0.0;
    }

    /* order key and its FP32 error bound */
    if (S->kind == 0) {
        G->zc = ms[2];
        G->tau = msmag[2];
        G->c[0] = G->WH[0][2] / G->WH[2][2];
        G->c[1] = G->WH[1][2] / G->WH[2][2];
    } else if (S->kind == 2) {
        /* cylinder: column from the azimuth about the camera's y axis, row
           from the height over the horizontal distance (pixel units) */
        G->zc = sqrt(ms[0] * ms[0] + ms[2] * ms[2]);
        G->tau = sqrt(msmag[0] * msmag[0] + msmag[2] * msmag[2]) + 3.0 * OR_U32 * G->zc;
        G->c[0] = S->cx + S->fx * atan2(ms[0], ms[2]);
        G->c[1] = S->cy + S->fy * ms[1] / G->zc;
    } else {
        G->zc = sqrt(or_dot3(ms, ms));
        G->tau = sqrt(or_dot3(msmag, msmag)) + 3.0 * OR_U32 * G->zc;
        double az = atan2(ms[1], ms[0]);
        double el = atan2(ms[2], sqrt(ms[0] * ms[0] + ms[1] * ms[1]));
        /* cell coordinates: ray (row i, column j) sits at (j, i) */
        G->c[0] = (az - S->az0) / S->d_az - 0.5;
        G->c[1] = (S->el_max - el) / S->d_el;
    }
    or_centre_error(G, S);
    G->culled = !(G->zc > S->near_);
    G->cull_rel = fabs(G->zc - S->near_) / S->near_;
    G->o = or_sigmoid(opacity_logit[i]);

    /* normal = third column of R, in the sensor frame, facing the sensor */
    double nw[3] = {R[0][2], R[1][2], R[2][2]};
    double to_s[3] = {mu[0] - S->origin[0], mu[1] - S->origin[1], mu[2] - S->origin[2]};
    double facing = or_dot3(nw, to_s);
    {
        /* error bound of the test in FP32: the differences mu - origin and
           the three-term dot product, each within gamma_4 of their terms */
        double terms = 0.0;
        for (int a = 0; a < 3; ++a) terms += fabs(nw[a]) * (fabs(mu[a]) + fabs(S->origin[a]) + mag[a]);
        G->n_amb = fabs(facing) <= OR_GAMMA4 * terms;
    }
    if (facing > 0) { nw[0] = -nw[0]; nw[1] = -nw[1]; nw[2] = -nw[2]; }
    for (int a = 0; a < 3; ++a) G->normal[a] = S->Rs[a][0] * nw[0] + S->Rs[a][1] * nw[1] + S->Rs[a][2] * nw[2];

    if (S->kind != 1) {
        double len = sqrt(or_dot3(to_s, to_s));
        double dw[3] = {to_s[0] / len, to_s[1] / len, to_s[2] / len};
        double dl[3]; /* into the object frame: R_o^T dw */
        for (int a = 0; a < 3; ++a) dl[a] = Ro[0][a] * dw[0] + Ro[1][a] * dw[1] + Ro[2][a] * dw[2];
        int K = (sh_degree + 1) * (sh_degree + 1);
        double col[3] = {0.5, 0.5, 0.5};
        int k = 0;
        for (int l = 0; l <= sh_degree; ++l)
            for (int m = -l; m <= l; ++m, ++k) {
                const double* c = sh + ((size_t)i * K + k) * 3;
                /* a band of exact zeros adds exact zeros: skip the basis */
                if (c[0] == 0.0 && c[1] == 0.0 && c[2] == 0.0) continue;
                double Y = oracle_sh_basis(l, m, dl);
                for (int ch = 0; ch < 3; ++ch) col[ch] += Y * c[ch];
            }
        for (int ch = 0; ch < 3; ++ch) G->feat[ch] = col[ch] > 0 ? col[ch] : 0.0;
    } else {
        G->feat[0] = intensity ? intensity[i] : 0.0;
        G->feat[1] = ray_drop ? or_sigmoid(ray_drop[i]) : 0.0; /* ray-drop probability rho */
        G->feat[2] = 0.0;
    }
}

/* ----------------------------------------------------------------------- */
/* Per-ray evaluation of one surfel                                          */
/* ----------------------------------------------------------------------- */
typedef struct {
    int idx;
    double zc;        /* centre depth: the order key */
    double alpha;     /* min(0.99, o G)       */
    double z;         /* contribution depth   */
    double rho3, rholp, zint;
    int v3, vlp;      /* support validity     */
    int hasplane;     /* m2 != 0              */
    int phantom;      /* culled by the near test, but within rounding of it */
    int use3;         /* the ray-splat intersection's weight won (else low-pass) */
    double uabs;      /* |u| + |v| of the intersection */
    double drholp;    /* bound on the change of rholp that the FP32 reach of
                         the low-pass centre (c_err) allows                 */
    double cosang;    /* |cos| of the angle between the ray and the surfel normal */
} or_hit;

/* k, l are the plane rows h_u^T WH, h_v^T WH; d (LiDAR only) the ray direction. */
static int or_eval(const or_surfel* G, const or_sensor* S, const double hu[4], const double hv[4],
                   const double d[3], const double pc[2], or_hit* h)
{
    double k[3], l[3], m[3];
    for (int b = 0; b < 3; ++b) {
        k[b] = hu[0] * G->WH[0][b] + hu[1] * G->WH[1][b] + hu[2] * G->WH[2][b] + hu[3] * G->WH[3][b];
        l[b] = hv[0] * G->WH[0][b] + hv[1] * G->WH[1][b] + hv[2] * G->WH[2][b] + hv[3] * G->WH[3][b];
    }
    /* Eq. 2: k . (u,v,1) = 0 and l . (u,v,1) = 0  =>  (u,v,1) ~ k x l */
    or_cross(k, l, m);
    h->hasplane = (m[2] != 0.0);
    h->v3 = 0;
    h->rho3 = INFINITY;
    h->zint = 0;
    h->uabs = 0;
    h->use3 = 0;
    if (h->hasplane) {
        double u = m[0] / m[2], v = m[1] / m[2];
        h->uabs = fabs(u) + fabs(v);
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = G->WH[a][0] * u + G->WH[a][1] * v + G->WH[a][2];
        double zi;
        if (S->kind == 0) zi = x[2];             /* depth row of W H        */
        else zi = or_dot3(x, d);                  /* LiDAR: distance along the unit ray;
                                                     cylinder: horizontal distance (d horizontal) */
        h->zint = zi;
        h->rho3 = u * u + v * v;
        h->v3 = (zi > S->near_) && (h->rho3 <= 9.0);
    }
    double dx = pc[0] - G->c[0], dy = pc[1] - G->c[1];
    if (S->kind == 1) { /* azimuth wraps around the spin */
        dx = fmod(dx, (double)S->columns);
        if (dx >= 0.5 * S->columns) dx -= S->columns;
        if (dx < -0.5 * S->columns) dx += S->columns;
    }
    h->rholp = (dx * dx + dy * dy) / 0.5; /* |p-c|^2 / sigma^2, sigma^2 = 1/2 */
    {
        double ex = G->c_err[0], ey = G->c_err[1];
        h->drholp = 4.0 * (fabs(dx) * ex + fabs(dy) * ey) + 2.0 * (ex * ex + ey * ey);
    }
    h->vlp = h->rholp <= 9.0;
    h->zc = G->zc;
    if (!h->v3 && !h->vlp) return 0;
    double rho;
    if (h->v3 && (!h->vlp || h->rho3 <= h->rholp)) { rho = h->rho3; h->z = h->zint; h->use3 = 1; }
    else { rho = h->rholp; h->z = G->zc; }
    double Gv = exp(-0.5 * rho);
    double a = G->o * Gv;
    h->alpha = a < 0.99 ? a : 0.99;
    return 1;
}

static double or_relm(double x, double thr) { return fabs(x - thr) / fabs(thr); }

/*
 * Whether surfel g enters ray's hit sequence, and its hit record.  A surfel
 * enters when it contributes a weight (or_eval), when one of its support
 * tests is within 1e-3 of its threshold (a near miss, whose acceptance an
 * FP32 evaluation could take the other way), or when it was culled by the
 * near test within rounding of the threshold (a phantom).
 */
static int or_collect(const or_surfel* g, int i, const or_sensor* S, const double hu[4], const double hv[4],
                      const double d[3], const double pc[2], const double dir[3], or_hit* h);

static int or_cmp_hit(const void* pa, const void* pb)
{
    const or_hit* a = (const or_hit*)pa;
    const or_hit* b = (const or_hit*)pb;
    if (a->zc < b->zc) return -1;
    if (a->zc > b->zc) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/*
 * Decisions that FP32 rounding could flip.  A threshold decision counts as
 * flippable when its relative distance to the threshold is below
 * OR_FLIP_REL (2e-5); the order of two contributing surfels counts as
 * flippable when their FP64 depths differ by less than the sum of their
 * FP32 error bounds (tau).  The recorded effect is the largest change of an
 * output that taking the decision the other way could cause (T times the
 * jump in alpha; for the depth-branch choice, the relative jump in depth
 * weight; for a near-tied run at the stop, the weight composited since the
 * run began; for a ray that meets a surfel at a glancing angle, the change of its
 * weight that the conditioning of Eq. 2 allows, see or_step).  A near-tied
 * run that composites whole does not flag the ray:
 * the change a reordering can make is bounded (or_run_close) and summed
 * into the ray's slack.
 */
#ifndef OR_FLIP_REL
#define OR_FLIP_REL 2e-5
#endif

/* Near-miss and phantom margin of or_collect (relative). */
#define OR_NEAR_MISS 1e-3

typedef struct {
    double feat[3], A, B, D, N[3], T;
    double flip;      /* largest effect of a flippable decision, 0 if none */
    double slack;     /* summed bound of the colour / intensity change a
                         reordering of near-tied runs can make             */
    double slack_n;   /* the same for the normal                           */
    double slack_z;   /* the same for sum w z (the depth accumulator B)    */
    double slack_c;   /* bound of the change of every output (relative
                         for depth) that FP32 rounding can cause through
                         the conditioning of Eq. 2 at glancing angles, or
                         by placing a near-tied hit before the stopping
                         surfel (or_after_stop)                            */
    int n_contrib;
    int done;         /* the stop rule ended the ray                       */
    /* the current run of near-tied composited surfels (consecutive centre
       depths within their FP32 error bounds of each other) */
    int run_len;
    double run_T0;                 /* T before the run's first surfel       */
    double last_zc, last_tau;      /* the run's last surfel                 */
    double lo[7], hi[7];           /* range of feat[3], normal[3], z        */
    const or_surfel* last_g;       /* the run's last surfel                 */
    double first_alpha, first_v[7], second_alpha, second_v[7];
    /* the surfel whose step ended the ray, and T there */
    const or_surfel* stop_g;
    double stop_zc, stop_tau, stop_T;
} or_ray;

static void or_flip(double* flip, double rel, double scale, double effect)
{
    if (rel < scale && effect > *flip) *flip = effect;
}

static void or_ray_init(or_ray* r)
{
    memset(r, 0, sizeof(*r));
    r->T = 1.0;
}

/*
 * Near-tied runs.  Two composited surfels whose FP64 centre depths differ by
 * less than the sum of their FP32 error bounds may come in either order
 * from an FP32 sort, and so may every surfel of a chain of such pairs.  The
 * composited weight of a run, T0 (1 - prod (1 - alpha_i)), does not depend
 * on its order, and neither does T after it, so under any order of the run
 * each output differs from the FP64 order's by at most the run's weight
 * times the range of that output over the run's surfels.  For a run of two
 * the change is exact: a swap moves alpha_1 alpha_2 T0 from one surfel's
 * value to the other's.
 */
static void or_run_close(or_ray* r)
{
    if (r->run_len >= 2) {
        double d[7];
        double W;
        if (r->run_len == 2) {
            W = r->first_alpha * r->second_alpha * r->run_T0;
            for (int c = 0; c < 7; ++c) d[c] = fabs(r->first_v[c] - r->second_v[c]);
        } else {
            W = r->run_T0 - r->T;
            for (int c = 0; c < 7; ++c) d[c] = r->hi[c] - r->lo[c];
        }
        double sf = d[0] > d[1] ? d[0] : d[1], sn = d[3] > d[4] ? d[3] : d[4];
        if (d[2] > sf) sf = d[2];
        if (d[5] > sn) sn = d[5];
        r->slack += W * sf;
        r->slack_n += W * sn;
        r->slack_z += W * d[6];
    }
    r->run_len = 0;
}

static void or_values(const or_surfel* g, const or_hit* h, double v[7])
{
    for (int c = 0; c < 3; ++c) {
        v[c] = g->feat[c];
        v[3 + c] = g->normal[c];
    }
    v[6] = h->z;
}

/* Finish a ray: close its last run. */
static void or_ray_finish(or_ray* r) { or_run_close(r); }

/*
 * One step of front-to-back compositing (3DGS order and thresholds): hit h
 * of surfel g is the next in depth order.  Accumulates sum w feat,
 * A = sum w, B = sum w z, D = sum w z^2 and sum w n, with w = alpha T, and
 * sets r->done when the stop rule ends the ray.
 */
/*
 * The conditioning of Eq. 2: where a ray meets the surfel plane at a
 * glancing angle, an FP32 rounding that moves the plane along its normal
 * (the centre's sensor-frame coordinates, each off by about u |mu_a|) or
 * turns the ray (LiDAR and cylinder rays come from rounded angles: about u
 * radians, times the distance t) moves the hit within the plane by that
 * amount over |cos|; in (u, v) units, over the scale.  Returns that bound of
 * |du| (and |dv|), 0 without an intersection.
 */
static double or_solve_error(const or_surfel* g, const or_hit* h, const or_sensor* S)
{
    if (!h->hasplane) return 0.0;
    double dn = 0.0;
    for (int a = 0; a < 3; ++a) dn += fabs(g->normal[a] * g->ms[a]);
    double turn = S->kind == 0 ? 0.0 : fabs(h->zint);
    return OR_SOLVE_ROUNDOFF * OR_U32 * (dn + turn) / (g->smin * (h->cosang > 1e-12 ? h->cosang : 1e-12));
}

static double or_max(double a, double b) { return a > b ? a : b; }

/* Two surfels whose FP32 keys are equal in any evaluation order (see
   key_exact): their tie is broken by index on both sides. */
static int or_same_key(const or_surfel* a, const or_surfel* b)
{
    return a->key_exact && b->key_exact && a->key_in[0] == b->key_in[0] && a->key_in[1] == b->key_in[1] &&
           a->key_in[2] == b->key_in[2];
}

static void or_step(or_ray* r, const or_surfel* g, const or_hit* h, const or_sensor* S)
{
    double T = r->T;
    /* the threshold margins: 2e-5 relative, or what the conditioning of the
       hit allows if that is more (u^2 + v^2 moves by 2 (|u| + |v|) du, alpha
       relatively by (|u| + |v|) du) */
    double du = or_solve_error(g, h, S);
    double m_rho = or_max(OR_FLIP_REL, 2.0 * h->uabs * du / 9.0);
    double m_alpha = h->use3 ? or_max(OR_FLIP_REL, h->uabs * du) : or_max(OR_FLIP_REL, 0.5 * h->drholp);
    double edge = T * g->o * exp(-4.5);
    if (h->hasplane && h->zint > S->near_) or_flip(&r->flip, or_relm(h->rho3, 9.0), m_rho, edge);
    if (h->hasplane && h->rho3 <= 9.0)
        or_flip(&r->flip, or_relm(h->zint, S->near_), OR_FLIP_REL, T * g->o * exp(-0.5 * h->rho3));
    or_flip(&r->flip, or_relm(h->rholp, 9.0), or_max(OR_FLIP_REL, h->drholp / 9.0), edge);
    if (h->alpha <= 0) return;
    /* the centre-depth cull of this surfel could go the other way */
    or_flip(&r->flip, g->cull_rel, OR_FLIP_REL, h->alpha * T);
    if (h->phantom) return;
    or_flip(&r->flip, or_relm(h->alpha, 1.0 / 255.0), m_alpha, T / 255.0);
    if (h->v3 && h->vlp) {
        double big = h->rho3 > h->rholp ? h->rho3 : h->rholp;
        or_flip(&r->flip, fabs(h->rho3 - h->rholp) / big,
                or_max(OR_FLIP_REL, (h->drholp + 2.0 * h->uabs * du) / big),
                h->alpha * T * fabs(h->zint - g->zc) / g->zc);
    }
    if (h->alpha < 1.0 / 255.0) return;
    double test = T * (1.0 - h->alpha);
    or_flip(&r->flip, or_relm(test, 1e-4), or_max(m_alpha * h->alpha / (1.0 - h->alpha), OR_FLIP_REL),
            h->alpha * T);
    /* a normal whose facing sign FP32 may take the other way: the normal
       output moves by twice its weight */
    if (g->n_amb && S->kind != 1) or_flip(&r->flip, 0.0, 1.0, 2.0 * h->alpha * T);
    /* the conditioning of Eq. 2 (or_solve_error): the weight follows the
       hit's (u, v) with alpha 0.5 d(u^2 + v^2) */
    if (h->use3 && h->alpha < 0.99) {
        double dalpha = h->alpha * h->uabs * du;
        /* this weight moves by T dalpha, the later ones by at most as much in
           all: a bound on each output's change, added to the ray's slack */
        r->slack_c += 2.0 * T * dalpha;
    } else if (!h->use3 && h->alpha < 0.99) {
        /* the low-pass weight moves relatively by half the reach of rholp */
        r->slack_c += T * h->alpha * h->drholp;
    }
    double v[7];
    or_values(g, h, v);
    int tie = r->run_len > 0 && fabs(h->zc - r->last_zc) <= g->tau + r->last_tau && !or_same_key(g, r->last_g);
    if (test < 1e-4) {
        /* reordered, the run could place this surfel before others of the
           run and stop the ray there instead: everything composited since
           the run began is at stake */
        if (tie) {
            double m = 1.0;
            for (int c = 0; c < 6; ++c) {
                if (fabs(v[c]) > m) m = fabs(v[c]);
                if (fabs(r->hi[c]) > m) m = fabs(r->hi[c]);
                if (fabs(r->lo[c]) > m) m = fabs(r->lo[c]);
            }
            or_flip(&r->flip, 0.0, 1.0, r->run_T0 * m);
        }
        r->done = 1;
        r->stop_g = g;
        r->stop_zc = h->zc;
        r->stop_tau = g->tau;
        r->stop_T = T;
        return;
    }
    if (!tie) {
        or_run_close(r);
        r->run_T0 = T;
        r->first_alpha = h->alpha;
        for (int c = 0; c < 7; ++c) r->lo[c] = r->hi[c] = r->first_v[c] = v[c];
    } else {
        if (r->run_len == 1) {
            r->second_alpha = h->alpha;
            for (int c = 0; c < 7; ++c) r->second_v[c] = v[c];
        }
        for (int c = 0; c < 7; ++c) {
            if (v[c] < r->lo[c]) r->lo[c] = v[c];
            if (v[c] > r->hi[c]) r->hi[c] = v[c];
        }
    }
    ++r->run_len;
    r->last_zc = h->zc;
    r->last_tau = g->tau;
    r->last_g = g;
    double w = h->alpha * T;
    for (int ch = 0; ch < 3; ++ch) r->feat[ch] += w * g->feat[ch];
    r->A += w;
    r->B += w * h->z;
    r->D += w * h->z * h->z;
    for (int a = 0; a < 3; ++a) r->N[a] += w * g->normal[a];
    r->T = test;
    ++r->n_contrib;
}

/*
 * Past the stop.  A hit after the stopping surfel in (depth, index) order
 * whose centre depth lies within the two FP32 error bounds of the stopping
 * surfel's may come before it from an FP32 sort.  There it composites
 * weight w = alpha T at the stop's T, and the ray still ends at the
 * stopping surfel (T only falls) or at this hit if it stops the ray itself.
 * So A and the final T move by w, a colour (with the background behind T)
 * by w |value - background|, the normal by w |n|, and the expected depth
 * B / A relatively by at most w |z / d - 1| for d = B / A at the stop.  The
 * largest of these, summed over such hits, is added to the ray's slack of
 * every output (slack_c).  Returns 0 once no later hit can be near-tied with
 * the stop: its depth is past the stop's by more than the stop's bound plus
 * tau_max, the largest bound of any surfel.
 */
static int or_after_stop(or_ray* r, const or_surfel* g, const or_hit* h, const or_sensor* S, double tau_max)
{
    if (h->zc - r->stop_zc > r->stop_tau + tau_max) return 0;
    if (h->alpha >= 1.0 / 255.0 && h->zc - r->stop_zc <= r->stop_tau + g->tau && !or_same_key(g, r->stop_g)) {
        double v[7];
        or_values(g, h, v);
        double m = 1.0;
        for (int c = 0; c < 3; ++c) m = or_max(m, fabs(v[c] - S->bg[c]));
        for (int c = 3; c < 6; ++c) m = or_max(m, fabs(v[c]));
        if (r->A > 0 && r->B > 0) m = or_max(m, fabs(v[6] * r->A / r->B - 1.0));
        r->slack_c += h->alpha * r->stop_T * m;
    }
    return 1;
}

static int or_collect(const or_surfel* g, int i, const or_sensor* S, const double hu[4], const double hv[4],
                      const double d[3], const double pc[2], const double dir[3], or_hit* h)
{
    if (g->culled && g->cull_rel >= OR_FLIP_REL) return 0;
    h->idx = i;
    h->phantom = g->culled;
    int any = or_eval(g, S, hu, hv, d, pc, h);
    h->cosang = fabs(or_dot3(g->normal, dir)) / sqrt(or_dot3(dir, dir));
    /* keep near misses too: their acceptance could flip in FP32 */
    int near_miss = (h->hasplane && h->zint > S->near_ && or_relm(h->rho3, 9.0) < OR_NEAR_MISS) ||
                    (h->hasplane && h->rho3 <= 9.0 && or_relm(h->zint, S->near_) < OR_NEAR_MISS) ||
                    or_relm(h->rholp, 9.0) < or_max(OR_NEAR_MISS, 2.0 * h->drholp / 9.0);
    if (!any && !near_miss) return 0;
    if (!any) { h->alpha = 0; h->z = g->zc; }
    return 1;
}

/* Brute force: every surfel against the ray, hits sorted by (depth, index). */
static void or_composite(const or_surfel* G, int n, const or_sensor* S, const double hu[4], const double hv[4],
                         const double d[3], const double pc[2], const double dir[3], double tau_max, or_hit* buf,
                         or_ray* out)
{
    int nh = 0;
    for (int i = 0; i < n; ++i)
        if (or_collect(&G[i], i, S, hu, hv, d, pc, dir, &buf[nh])) ++nh;
    qsort(buf, (size_t)nh, sizeof(or_hit), or_cmp_hit);
    or_ray_init(out);
    int j = 0;
    for (; j < nh && !out->done; ++j) or_step(out, &G[buf[j].idx], &buf[j], S);
    if (out->done)
        for (; j < nh && or_after_stop(out, &G[buf[j].idx], &buf[j], S, tau_max); ++j) {}
    or_ray_finish(out);
}

/* ----------------------------------------------------------------------- */
/* Tiled mode: the same compositing over per-tile candidate lists.           */
/* ----------------------------------------------------------------------- */
/*
 * A ray-index box [x0, x1] x [y0, y1] (inclusive, in pixel or LiDAR cell
 * coordinates of ray centres) holding every ray that surfel g could enter
 * (or_collect), including near misses and phantoms.  Returns 0 if no ray
 * can see it, 1 otherwise; *all_x / *all_y ask for the whole axis.
 *
 * The bound is the oracle's own, written from the geometry: the support
 * u^2 + v^2 <= 9 (with the near-miss margin) lies inside the square of
 * half-width 3.01 s in the surfel plane, and inside the sphere of radius
 * 3.01 max(s_u, s_v) about the centre; the low-pass disc lies within 2.13
 * pixels (cells) of the projected centre, plus six times the centre's FP32
 * reach (c_err).
 *   pinhole   -- the square clipped to the half-space in front of the near
 *                plane (where an intersection can count), projected: a
 *                convex polygon in front of the camera projects inside the
 *                convex hull of its projected vertices;
 *   cylinder  -- the sphere's azimuth cone asin(r / r_h) and its height
 *                ratio y / r_h over the sphere's box, else every pixel;
 *   LiDAR     -- the sphere's cap of angular radius beta = asin(r / |mu|):
 *                elevation +- beta, azimuth +- asin(sin(beta) / cos(el))
 *                (every column when the cap reaches a pole).
 * A phantom (culled within rounding of the near test) sees every ray.
 */
static int or_bound(const or_surfel* g, const or_sensor* S, double box[4], int* all_x, int* all_y)
{
    *all_x = *all_y = 0;
    if (g->culled) {
        if (g->cull_rel >= OR_FLIP_REL) return 0;
        *all_x = *all_y = 1;
        return 1;
    }
    /* 3 sigma_lp with the near-miss margin, and more; widened by six times
       the centre's FP32 reach, which holds every rholp <= 9 + 2 drholp */
    const double lp = 2.13 + 6.0 * or_max(g->c_err[0], g->c_err[1]);
    double x0 = g->c[0] - lp, x1 = g->c[0] + lp, y0 = g->c[1] - lp, y1 = g->c[1] + lp;
    const double* m = g->ms;
    const double r = g->rad;
    if (S->kind == 0) {
        /* the half-width 3.01 square in (u, v), clipped to the half-plane
           where the intersection depth can pass the near test (depth is
           affine in u, v), then projected through W H: a convex polygon in
           front of the camera projects inside the convex hull of its
           projected vertices */
        double zmin = S->near_ * (1.0 - 2.0 * OR_NEAR_MISS);
        double sq[4][2] = {{-3.01, -3.01}, {3.01, -3.01}, {3.01, 3.01}, {-3.01, 3.01}};
        double poly[8][2];
        int np_ = 0;
        for (int k = 0; k < 4; ++k) {
            const double* a = sq[k];
            const double* b = sq[(k + 1) & 3];
            double za = g->WH[2][0] * a[0] + g->WH[2][1] * a[1] + g->WH[2][2] - zmin;
            double zb = g->WH[2][0] * b[0] + g->WH[2][1] * b[1] + g->WH[2][2] - zmin;
            if (za >= 0) { poly[np_][0] = a[0]; poly[np_][1] = a[1]; ++np_; }
            if ((za >= 0) != (zb >= 0)) {
                double t = za / (za - zb);
                poly[np_][0] = a[0] + t * (b[0] - a[0]);
                poly[np_][1] = a[1] + t * (b[1] - a[1]);
                ++np_;
            }
        }
        for (int k = 0; k < np_; ++k) {
            double u = poly[k][0], v = poly[k][1];
            double X = g->WH[0][0] * u + g->WH[0][1] * v + g->WH[0][2];
            double Y = g->WH[1][0] * u + g->WH[1][1] * v + g->WH[1][2];
            double Z = g->WH[2][0] * u + g->WH[2][1] * v + g->WH[2][2];
            if (!(Z > 0.5 * zmin)) { *all_x = *all_y = 1; return 1; } /* rounding at the clip */
            double px = X / Z, py = Y / Z;
            if (px < x0) x0 = px;
            if (px > x1) x1 = px;
            if (py < y0) y0 = py;
            if (py > y1) y1 = py;
        }
    } else if (S->kind == 2) {
        double rh = g->zc;
        if (!(rh - r > S->near_)) { *all_x = *all_y = 1; return 1; }
        double az = atan2(m[0], m[2]), daz = asin(r / rh);
        if (az - daz <= -OR_PI || az + daz >= OR_PI) *all_x = 1;
        double ax0 = S->cx + S->fx * (az - daz), ax1 = S->cx + S->fx * (az + daz);
        double ylo = m[1] - r, yhi = m[1] + r, rlo = rh - r, rhi = rh + r;
        double q[4] = {ylo / rlo, ylo / rhi, yhi / rlo, yhi / rhi};
        double q0 = q[0], q1 = q[0];
        for (int k = 1; k < 4; ++k) {
            if (q[k] < q0) q0 = q[k];
            if (q[k] > q1) q1 = q[k];
        }
        if (ax0 < x0) x0 = ax0;
        if (ax1 > x1) x1 = ax1;
        if (S->cy + S->fy * q0 < y0) y0 = S->cy + S->fy * q0;
        if (S->cy + S->fy * q1 > y1) y1 = S->cy + S->fy * q1;
    } else {
        double rng = g->zc;
        if (!(rng - r > S->near_)) { *all_x = *all_y = 1; return 1; }
        double beta = asin(r / rng);
        double el = atan2(m[2], sqrt(m[0] * m[0] + m[1] * m[1]));
        double az = atan2(m[1], m[0]);
        double ey0 = (S->el_max - (el + beta)) / S->d_el, ey1 = (S->el_max - (el - beta)) / S->d_el;
        if (ey0 < y0) y0 = ey0;
        if (ey1 > y1) y1 = ey1;
        double sa = sin(beta) / cos(el);
        if (fabs(el) + beta >= 0.5 * OR_PI || !(sa < 1.0)) *all_x = 1;
        else {
            double daz = asin(sa);
            double ex0 = (az - daz - S->az0) / S->d_az - 0.5, ex1 = (az + daz - S->az0) / S->d_az - 0.5;
            if (ex0 < x0) x0 = ex0;
            if (ex1 > x1) x1 = ex1;
        }
    }
    /* one more ray of margin against rounding in the bound itself */
    box[0] = x0 - 1.0; box[1] = x1 + 1.0; box[2] = y0 - 1.0; box[3] = y1 + 1.0;
    return 1;
}

typedef struct {
    double zc;
    int idx;
} or_cand;

static int or_cmp_cand(const void* pa, const void* pb)
{
    const or_cand* a = (const or_cand*)pa;
    const or_cand* b = (const or_cand*)pb;
    if (a->zc < b->zc) return -1;
    if (a->zc > b->zc) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/*
 * Per-tile candidate lists: tile (tx, ty) of tile x tile rays holds every
 * surfel whose or_bound box meets one of its ray centres, sorted by
 * (depth, index).  Ray (x, y) -- pixel column/row, or LiDAR column/beam --
 * has its centre at (x + 0.5, y + 0.5) for the cameras and at (x, y) in the
 * LiDAR's cell coordinates; LiDAR columns wrap.  Returns 0 on success.
 */
typedef struct {
    int tile, tiles_x, tiles_y, nx, ny;
    long long* start;   /* [tiles + 1] */
    or_cand* cand;
} or_tiles;

static void or_box_tiles(const or_sensor* S, const or_tiles* T, const double box[4], int all_x, int all_y,
                         int* tx0, int* tx1, int* ty0, int* ty1, int* wrap)
{
    /* ray centre offset along each axis: cameras at +0.5, LiDAR cells at 0 */
    double off = (S->kind == 1) ? 0.0 : 0.5;
    *wrap = 0;
    if (all_y) { *ty0 = 0; *ty1 = T->ny - 1; }
    else {
        double a = ceil(box[2] - off), b = floor(box[3] - off);
        if (a < 0) a = 0;
        if (b > T->ny - 1) b = T->ny - 1;
        *ty0 = (int)a; *ty1 = (int)b;
    }
    if (all_x || (S->kind == 1 && box[1] - box[0] >= T->nx - 1)) { *tx0 = 0; *tx1 = T->nx - 1; }
    else {
        double a = ceil(box[0] - off), b = floor(box[1] - off);
        if (S->kind == 1) {
            /* columns on the circle: shift the interval so it starts in range */
            double sh = floor(a / T->nx) * T->nx;
            a -= sh; b -= sh;
            if (b > T->nx - 1) *wrap = 1; /* [a, nx) and [0, b - nx] */
        } else {
            if (a < 0) a = 0;
            if (b > T->nx - 1) b = T->nx - 1;
        }
        *tx0 = (int)a; *tx1 = (int)b;
    }
    /* to tiles */
    if (*ty0 <= *ty1) { *ty0 /= T->tile; *ty1 /= T->tile; }
    if (*wrap) {
        *tx1 = (*tx1 - T->nx) / T->tile; /* second piece [0, tx1] */
        *tx0 /= T->tile;                 /* first piece [tx0, tiles_x) */
    } else if (*tx0 <= *tx1) { *tx0 /= T->tile; *tx1 /= T->tile; }
}

static void or_tiles_free(or_tiles* T)
{
    free(T->start);
    free(T->cand);
    T->start = NULL;
    T->cand = NULL;
}

static int or_tiles_build(or_tiles* T, const or_surfel* G, int n, const or_sensor* S, int tile, int nx, int ny)
{
    T->tile = tile;
    T->nx = nx;
    T->ny = ny;
    T->tiles_x = (nx + tile - 1) / tile;
    T->tiles_y = (ny + tile - 1) / tile;
    long long nt = (long long)T->tiles_x * T->tiles_y;
    T->start = (long long*)calloc((size_t)nt + 1, sizeof(long long));
    T->cand = NULL;
    int* rect = (int*)malloc(sizeof(int) * 5 * (size_t)(n > 0 ? n : 1));
    long long* cnt = (long long*)calloc((size_t)nt, sizeof(long long));
    if (!T->start || !rect || !cnt) { free(rect); free(cnt); or_tiles_free(T); return -1; }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double box[4];
        int ax, ay;
        int* R = rect + 5 * i;
        if (!or_bound(&G[i], S, box, &ax, &ay)) { R[0] = 1; R[1] = 0; R[2] = 1; R[3] = 0; R[4] = 0; continue; }
        or_box_tiles(S, T, box, ax, ay, &R[0], &R[1], &R[2], &R[3], &R[4]);
    }
    /* count, then fill (in any order: each list is sorted afterwards by
       (depth, index), a total order, so the result does not depend on it) */
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 1024)
        for (int i = 0; i < n; ++i) {
            const int* R = rect + 5 * i;
            if (R[2] > R[3]) continue;
            for (int ty = R[2]; ty <= R[3]; ++ty) {
                long long row = (long long)ty * T->tiles_x;
                int pieces = R[4] ? 2 : 1;
                for (int p = 0; p < pieces; ++p) {
                    int a = R[4] ? (p == 0 ? R[0] : 0) : R[0];
                    int b = R[4] ? (p == 0 ? T->tiles_x - 1 : R[1]) : R[1];
                    if (R[4] && p == 1 && b >= R[0]) b = R[0] - 1; /* pieces overlap: whole row once */
                    for (int tx = a; tx <= b; ++tx) {
                        if (pass == 0) {
#pragma omp atomic
                            ++cnt[row + tx];
                        } else {
                            long long at;
#pragma omp atomic capture
                            at = cnt[row + tx]++;
                            at += T->start[row + tx];
                            T->cand[at].zc = G[i].zc;
                            T->cand[at].idx = i;
                        }
                    }
                }
            }
        }
        if (pass == 0) {
            for (long long t = 0; t < nt; ++t) T->start[t + 1] = T->start[t] + cnt[t];
            memset(cnt, 0, sizeof(long long) * (size_t)nt);
            T->cand = (or_cand*)malloc(sizeof(or_cand) * (size_t)(T->start[nt] > 0 ? T->start[nt] : 1));
            if (!T->cand) { free(rect); free(cnt); or_tiles_free(T); return -1; }
        }
    }
    free(rect);
    free(cnt);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < nt; ++t)
        qsort(T->cand + T->start[t], (size_t)(T->start[t + 1] - T->start[t]), sizeof(or_cand), or_cmp_cand);
    return 0;
}

/*
 * Whether the ray (the line through the sensor origin along `dir`, sensor
 * frame) can reach surfel g: it passes within g->rad of the centre (the
 * sphere that holds the support with its near-miss margin), or the ray's
 * low-pass centre lies within 2.13 pixels (cells), plus six times the
 * centre's FP32 reach, of the surfel's.  A
 * surfel for which both fail is neither a hit nor a near miss of this ray
 * (or_collect would drop it), so the tiled walk may skip it.
 */
static int or_ray_may_reach(const or_surfel* g, const or_sensor* S, const double dir[3], double dir2,
                            const double pc[2])
{
    if (g->culled) return 1;
    double dx = pc[0] - g->c[0], dy = pc[1] - g->c[1];
    if (S->kind == 1) {
        dx = fmod(dx, (double)S->columns);
        if (dx >= 0.5 * S->columns) dx -= S->columns;
        if (dx < -0.5 * S->columns) dx += S->columns;
    }
    double lp = 2.13 + 6.0 * or_max(g->c_err[0], g->c_err[1]);
    if (dx * dx + dy * dy <= lp * lp) return 1;
    double c[3];
    or_cross(g->ms, dir, c);
    /* squared distance of the centre from the line: |m x d|^2 / |d|^2 */
    return or_dot3(c, c) <= g->rad * g->rad * dir2 * (1.0 + 1e-9);
}

/* The tiled walk of one ray: its tile's candidates in (depth, index) order. */
static void or_composite_tiled(const or_surfel* G, const or_tiles* T, long long tile_id, const or_sensor* S,
                               const double hu[4], const double hv[4], const double d[3], const double pc[2],
                               const double dir[3], double tau_max, or_ray* out)
{
    double dir2 = or_dot3(dir, dir);
    or_ray_init(out);
    long long q = T->start[tile_id];
    for (; q < T->start[tile_id + 1] && !out->done; ++q) {
        int i = T->cand[q].idx;
        if (!or_ray_may_reach(&G[i], S, dir, dir2, pc)) continue;
        or_hit h;
        if (or_collect(&G[i], i, S, hu, hv, d, pc, dir, &h)) or_step(out, &G[i], &h, S);
    }
    /* past the stop: the same hits in the same order as the brute-force walk */
    for (; out->done && q < T->start[tile_id + 1]; ++q) {
        int i = T->cand[q].idx;
        if (T->cand[q].zc - out->stop_zc > out->stop_tau + tau_max) break;
        if (!or_ray_may_reach(&G[i], S, dir, dir2, pc)) continue;
        or_hit h;
        if (or_collect(&G[i], i, S, hu, hv, d, pc, dir, &h) && !or_after_stop(out, &G[i], &h, S, tau_max))
            break;
    }
    or_ray_finish(out);
}

static or_surfel* or_prepare_all(int n, const or_sensor* S, const double* pos, const double* log_scale,
                                 const double* quat, const double* opacity_logit, int sh_degree,
                                 const double* sh, const double* intensity, const double* ray_drop,
                                 const int* obj_id, const double* obj_pose)
{
    or_surfel* G = (or_surfel*)malloc(sizeof(or_surfel) * (size_t)(n > 0 ? n : 1));
    if (!G) return NULL;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        or_prepare(&G[i], i, S, pos, log_scale, quat, opacity_logit, sh_degree, sh, intensity, ray_drop, obj_id,
                   obj_pose);
    return G;
}

/*
 * One ray of a sensor: its two planes (Eq. 3, 4 or 5), the direction used
 * for the depth of an intersection, and its low-pass centre.  (x, y) is the
 * pixel column/row, or the LiDAR column/beam.
 */
static void or_ray_planes(const or_sensor* S, int x, int y, double hu[4], double hv[4], double d[3], double pc[2],
                          double dir[3])
{
    if (S->kind == 0) {
        double px = x + 0.5, py = y + 0.5;
        hu[0] = -1; hu[1] = 0; hu[2] = 0; hu[3] = px; /* Eq. 3 */
        hv[0] = 0; hv[1] = -1; hv[2] = 0; hv[3] = py;
        d[0] = 0; d[1] = 0; d[2] = 1;
        pc[0] = px; pc[1] = py;
        dir[0] = (px - S->cx) / S->fx; dir[1] = (py - S->cy) / S->fy; dir[2] = 1.0;
    } else if (S->kind == 2) {
        double px = x + 0.5, py = y + 0.5;
        double phi = (px - S->cx) / S->fx, yn = (py - S->cy) / S->fy;
        hu[0] = cos(phi); hu[1] = 0; hu[2] = -sin(phi); hu[3] = 0; /* Eq. 4 */
        hv[0] = yn * sin(phi); hv[1] = -1; hv[2] = yn * cos(phi); hv[3] = 0;
        d[0] = sin(phi); d[1] = 0; d[2] = cos(phi); /* horizontal part of the ray */
        pc[0] = px; pc[1] = py;
        dir[0] = sin(phi); dir[1] = yn; dir[2] = cos(phi);
    } else {
        double el = S->el_max - y * S->d_el;
        double az = S->az0 + (x + 0.5) * S->d_az;
        hu[0] = sin(az); hu[1] = -cos(az); hu[2] = 0; hu[3] = 0; /* Eq. 5 */
        hv[0] = sin(el) * cos(az); hv[1] = sin(el) * sin(az); hv[2] = -cos(el); hv[3] = 0;
        d[0] = cos(el) * cos(az); d[1] = cos(el) * sin(az); d[2] = sin(el);
        pc[0] = (double)x; pc[1] = (double)y;
        dir[0] = d[0]; dir[1] = d[1]; dir[2] = d[2];
    }
}

/*
 * Every listed ray of a sensor (pix == NULL: all nx * ny rays, row-major),
 * brute force (tile == 0) or over per-tile lists (tile > 0); the same
 * compositing either way.  emit(q, ray, ctx) stores ray q's outputs.
 */
typedef void (*or_emit_fn)(long long q, const or_ray* r, void* ctx);

static int or_render_rays(const or_surfel* G, int n, const or_sensor* S, int nx, int ny, long long nq,
                          const long long* pix, int tile, or_emit_fn emit, void* ctx)
{
    int fail = 0;
    double tau_max = 0.0;
    for (int i = 0; i < n; ++i)
        if (G[i].tau > tau_max) tau_max = G[i].tau;
    if (tile > 0) {
        or_tiles T;
        if (or_tiles_build(&T, G, n, S, tile, nx, ny) != 0) return -1;
#pragma omp parallel for schedule(dynamic, 64)
        for (long long q = 0; q < nq; ++q) {
            long long li = pix ? pix[q] : q;
            int x = (int)(li % nx), y = (int)(li / nx);
            double hu[4], hv[4], d[3], pc[2], dir[3];
            or_ray_planes(S, x, y, hu, hv, d, pc, dir);
            or_ray r;
            or_composite_tiled(G, &T, (long long)(y / tile) * T.tiles_x + x / tile, S, hu, hv, d, pc, dir, tau_max,
                               &r);
            emit(q, &r, ctx);
        }
        or_tiles_free(&T);
        return 0;
    }
#pragma omp parallel
    {
        or_hit* buf = (or_hit*)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (long long q = 0; q < nq; ++q) {
                long long li = pix ? pix[q] : q;
                int x = (int)(li % nx), y = (int)(li / nx);
                double hu[4], hv[4], d[3], pc[2], dir[3];
                or_ray_planes(S, x, y, hu, hv, d, pc, dir);
                or_ray r;
                or_composite(G, n, S, hu, hv, d, pc, dir, tau_max, buf, &r);
                emit(q, &r, ctx);
            }
            free(buf);
        }
    }
    return fail ? -1 : 0;
}

typedef struct {
    const double* bg;
    double *rgb, *depth, *normal, *alpha, *trans, *acc, *flip, *slack;
    int* n_contrib;
} or_cam_out;

static void or_emit_camera(long long q, const or_ray* r, void* ctx)
{
    or_cam_out* o = (or_cam_out*)ctx;
    for (int ch = 0; ch < 3; ++ch) o->rgb[q * 3 + ch] = r->feat[ch] + r->T * o->bg[ch];
    o->depth[q] = r->A > 0 ? r->B / r->A : 0.0;
    for (int a = 0; a < 3; ++a) o->normal[q * 3 + a] = r->N[a];
    o->alpha[q] = r->A;
    o->trans[q] = r->T;
    if (o->acc) { o->acc[q * 3 + 0] = r->A; o->acc[q * 3 + 1] = r->B; o->acc[q * 3 + 2] = r->D; }
    if (o->flip) o->flip[q] = r->flip;
    if (o->slack) {
        o->slack[q * 4 + 0] = r->slack;
        o->slack[q * 4 + 1] = r->slack_n;
        o->slack[q * 4 + 2] = r->slack_z;
        o->slack[q * 4 + 3] = r->slack_c;
    }
    if (o->n_contrib) o->n_contrib[q] = r->n_contrib;
}

static int or_render_camera(int kind, int n, const double* pos, const double* log_scale, const double* quat,
                            const double* opacity_logit, int sh_degree, const double* sh,
                            const int* obj_id, const double* obj_pose,
                            int width, int height, double fx, double fy, double cx, double cy,
                            double near_, const double* world_to_cam, const double* bg,
                            int n_pix, const long long* pix, int tile,
                            double* rgb, double* depth, double* normal, double* alpha, double* trans,
                            double* acc, double* flip, double* slack, int* n_contrib)
{
    if (n < 0 || width <= 0 || height <= 0 || sh_degree < 0 || sh_degree > 3 || tile < 0) return -1;
    or_sensor S;
    memset(&S, 0, sizeof(S));
    S.kind = kind;
    or_sensor_from_matrix(&S, world_to_cam);
    S.fx = fx; S.fy = fy; S.cx = cx; S.cy = cy; S.near_ = near_;
    for (int c = 0; c < 3; ++c) S.bg[c] = bg[c];
    S.width = width; S.height = height;
    or_surfel* G = or_prepare_all(n, &S, pos, log_scale, quat, opacity_logit, sh_degree, sh, NULL, NULL, obj_id, obj_pose);
    if (!G) return -1;
    long long npx = pix ? n_pix : (long long)width * height;
    or_cam_out o = {bg, rgb, depth, normal, alpha, trans, acc, flip, slack, n_contrib};
    int rc = or_render_rays(G, n, &S, width, height, npx, pix, tile, or_emit_camera, &o);
    free(G);
    return rc;
}

/*
 * Pinhole camera frame (Eq. 3).  Pixel (x, y) has centre (x+0.5, y+0.5).
 * pix == NULL renders every pixel (n_pix = width*height, row-major), else
 * the n_pix listed pixels y*width+x.  Outputs are pixel-major:
 * rgb/normal [n_pix][3], the rest [n_pix].  rgb includes bg*T; depth is
 * sum(w z)/sum(w) (0 where sum(w) == 0); normal is sum(w n), unnormalised;
 * acc = [sum w, sum w z, sum w z^2] per pixel ([n_pix][3], may be NULL).
 * flip [n_pix] is the largest output change an FP32-flippable threshold
 * decision could cause (0 if none); slack [n_pix][4] bounds the change a
 * reordering of near-tied surfels can make to colour, to the normal and to
 * sum w z, and (fourth) the change of any output that FP32 rounding can
 * cause through the conditioning of Eq. 2 (both may be NULL).
 * tile == 0 checks every surfel for every pixel (brute force); tile > 0
 * walks per-tile candidate lists of tile x tile pixels built from the
 * oracle's own conservative bound, with the same arithmetic and the same
 * results.  Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_render_pinhole(int n, const double* pos, const double* log_scale, const double* quat,
                          const double* opacity_logit, int sh_degree, const double* sh,
                          const int* obj_id, const double* obj_pose,
                          int width, int height, double fx, double fy, double cx, double cy,
                          double near_, const double* world_to_cam, const double* bg,
                          int n_pix, const long long* pix, int tile,
                          double* rgb, double* depth, double* normal, double* alpha, double* trans,
                          double* acc, double* flip, double* slack, int* n_contrib)
{
    return or_render_camera(0, n, pos, log_scale, quat, opacity_logit, sh_degree, sh, obj_id, obj_pose, width,
                            height, fx, fy, cx, cy, near_, world_to_cam, bg, n_pix, pix, tile, rgb, depth, normal,
                            alpha, trans, acc, flip, slack, n_contrib);
}

/*
 * Cylindrical camera frame (Eq. 4): pixel (x, y) has
 * azimuth phi = (x + 0.5 - cx)/fx about the camera's y axis and height
 * y_n = (y + 0.5 - cy)/fy on the unit cylinder, so its ray from the camera
 * centre is d = (sin phi, y_n, cos phi).  The paper's h_u = (cos phi, 0,
 * -sin phi, 0) contains it; its printed h_v = (0, -1, 0, p_y) is a
 * pixel-frame row next to a camera-frame h_u, so h_v is read as the plane
 * through the camera centre that contains d and the horizontal direction
 * (cos phi, 0, -sin phi): h_v = (y_n sin phi, -1, y_n cos phi, 0), normal to
 * h_u as the paper's two planes are.  Depth is the horizontal distance t of
 * the intersection t d (the cylinder radius).
 * Outputs and `tile` as oracle_render_pinhole.
 */
int oracle_render_cylindrical(int n, const double* pos, const double* log_scale, const double* quat,
                              const double* opacity_logit, int sh_degree, const double* sh,
                              const int* obj_id, const double* obj_pose,
                              int width, int height, double fx, double fy, double cx, double cy,
                              double near_, const double* world_to_cam, const double* bg,
                              int n_pix, const long long* pix, int tile,
                              double* rgb, double* depth, double* normal, double* alpha, double* trans,
                              double* acc, double* flip, double* slack, int* n_contrib)
{
    return or_render_camera(2, n, pos, log_scale, quat, opacity_logit, sh_degree, sh, obj_id, obj_pose, width,
                            height, fx, fy, cx, cy, near_, world_to_cam, bg, n_pix, pix, tile, rgb, depth, normal,
                            alpha, trans, acc, flip, slack, n_contrib);
}

typedef struct {
    double *range, *intens, *drop, *alpha, *trans, *flip, *slack;
    int* n_contrib;
} or_lidar_out;

static void or_emit_lidar(long long q, const or_ray* r, void* ctx)
{
    or_lidar_out* o = (or_lidar_out*)ctx;
    o->range[q] = r->A > 0 ? r->B / r->A : 0.0;
    o->intens[q] = r->feat[0];
    if (o->drop) o->drop[q] = r->feat[1] + r->T;
    o->alpha[q] = r->A;
    o->trans[q] = r->T;
    if (o->flip) o->flip[q] = r->flip;
    if (o->slack) {
        o->slack[q * 4 + 0] = r->slack;
        o->slack[q * 4 + 1] = r->slack_n;
        o->slack[q * 4 + 2] = r->slack_z;
        o->slack[q * 4 + 3] = r->slack_c;
    }
    if (o->n_contrib) o->n_contrib[q] = r->n_contrib;
}

/*
 * Spinning LiDAR range image (Eq. 5).  Row i (beam) has elevation
 * el_max - i (el_max - el_min)/(beams-1); column j has azimuth
 * az0 + (j+0.5) 360/columns.  Outputs per ray: range = sum(w t)/sum(w)
 * (0 where sum(w) == 0), intensity = sum(w r), acc = sum(w), T, and the
 * ray-drop probability sum(w rho) + T with rho = sigmoid(ray_drop logit)
 * of each surfel (Sec. III-A lists rho among the LiDAR scene's attributes;
 * composited like the intensity, a ray that leaves the scene returns
 * nothing).  ray_drop may be NULL (rho = 0).  `tile`, flip and slack as
 * for the cameras (tiles of tile beams x tile columns; columns wrap; the
 * slack's first value covers intensity and ray drop).
 */
int oracle_render_lidar(int n, const double* pos, const double* log_scale, const double* quat,
                        const double* opacity_logit, const double* intensity, const double* ray_drop,
                        const int* obj_id, const double* obj_pose,
                        int beams, int columns, double el_min_deg, double el_max_deg, double az0_deg,
                        double near_, const double* world_to_lidar,
                        int n_ray, const long long* ray, int tile,
                        double* range, double* intens, double* drop, double* alpha, double* trans, double* flip,
                        double* slack, int* n_contrib)
{
    if (n < 0 || beams < 2 || columns <= 0 || tile < 0) return -1;
    or_sensor S;
    memset(&S, 0, sizeof(S));
    S.kind = 1;
    or_sensor_from_matrix(&S, world_to_lidar);
    S.beams = beams; S.columns = columns;
    S.el_max = el_max_deg * OR_PI / 180.0;
    S.d_el = (el_max_deg - el_min_deg) * OR_PI / 180.0 / (beams - 1);
    S.az0 = az0_deg * OR_PI / 180.0;
    S.d_az = 2.0 * OR_PI / columns;
    S.near_ = near_;
    or_surfel* G = or_prepare_all(n, &S, pos, log_scale, quat, opacity_logit, 0, NULL, intensity, ray_drop, obj_id,
                                  obj_pose);
    if (!G) return -1;
    long long nr = ray ? n_ray : (long long)beams * columns;
    or_lidar_out o = {range, intens, drop, alpha, trans, flip, slack, n_contrib};
    int rc = or_render_rays(G, n, &S, columns, beams, nr, ray, tile, or_emit_lidar, &o);
    free(G);
    return rc;
}

/* Number of threads the OpenMP runtime will use (for the benchmark report). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Eq. 2 for one surfel and one pixel / ray, exposed for the pins: returns
 * 1 and (u, v, depth-or-distance) if k x l has a non-zero third component.
 * kind 0 = pinhole (ray = pixel centre px,py), 1 = LiDAR (ray = az, el in
 * radians), 2 = cylinder (ray = azimuth phi, height y_n).  cam = {fx, fy,
 * cx, cy} for the cameras.
 */
int oracle_intersect(int kind, const double* pos, const double* log_scale, const double* quat,
                     const double* world_to_sensor, const double* cam, double a, double b, double* uvz)
{
    or_sensor S;
    memset(&S, 0, sizeof(S));
    S.kind = kind;
    or_sensor_from_matrix(&S, world_to_sensor);
    if (kind != 1) { S.fx = cam[0]; S.fy = cam[1]; S.cx = cam[2]; S.cy = cam[3]; }
    S.near_ = -1e300;
    S.columns = 1;
    double op = 0.0, ones = 0.0;
    or_surfel G;
    or_prepare(&G, 0, &S, pos, log_scale, quat, &op, 0, &ones, NULL, NULL, NULL, NULL);
    double hu[4], hv[4], d[3] = {0, 0, 1}, pc[2] = {0, 0};
    if (kind == 0) {
        hu[0] = -1; hu[1] = 0; hu[2] = 0; hu[3] = a;
        hv[0] = 0; hv[1] = -1; hv[2] = 0; hv[3] = b;
    } else if (kind == 2) { /* a = azimuth phi, b = height y_n on the unit cylinder */
        hu[0] = cos(a); hu[1] = 0; hu[2] = -sin(a); hu[3] = 0;
        hv[0] = b * sin(a); hv[1] = -1; hv[2] = b * cos(a); hv[3] = 0;
        d[0] = sin(a); d[1] = 0; d[2] = cos(a);
    } else {
        hu[0] = sin(a); hu[1] = -cos(a); hu[2] = 0; hu[3] = 0;
        hv[0] = sin(b) * cos(a); hv[1] = sin(b) * sin(a); hv[2] = -cos(b); hv[3] = 0;
        d[0] = cos(b) * cos(a); d[1] = cos(b) * sin(a); d[2] = sin(b);
    }
    or_hit h;
    or_eval(&G, &S, hu, hv, d, pc, &h);
    if (!h.hasplane) return 0;
    uvz[2] = h.zint;
    /* signed u, v from k x l */
    {
        double k[3], l[3], m[3];
        for (int c = 0; c < 3; ++c) {
            k[c] = hu[0] * G.WH[0][c] + hu[1] * G.WH[1][c] + hu[2] * G.WH[2][c] + hu[3] * G.WH[3][c];
            l[c] = hv[0] * G.WH[0][c] + hv[1] * G.WH[1][c] + hv[2] * G.WH[2][c] + hv[3] * G.WH[3][c];
        }
        or_cross(k, l, m);
        uvz[0] = m[0] / m[2];
        uvz[1] = m[1] / m[2];
    }
    return 1;
}
