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
 *   - composite order: centre depth (camera z, LiDAR |mu|), ties by index,
 *     with the depth key and the near cull taken in the kernel's FP32
 *     arithmetic (see or_key32);
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
    int culled;
    double WH[4][3];   /* Eq. 1: W . H, a 4x3 matrix                         */
    double zc;         /* centre depth (camera z) / centre range (LiDAR |mu|) */
    float key;         /* composite-order key: zc in the kernel's FP32 arithmetic */
    double c[2];       /* low-pass centre (pixels, or LiDAR cells)           */
    double o;          /* opacity, sigmoid of the logit                      */
    double feat[3];    /* camera: colour; LiDAR: intensity, ray drop, 0     */
    double normal[3];  /* sensor frame, facing the sensor                    */
} or_surfel;

typedef struct {
    /* sensor */
    int kind;                        /* 0 pinhole, 1 LiDAR, 2 cylindrical   */
    double Rs[3][3], ts[3];          /* world -> sensor rigid part          */
    double origin[3];                /* sensor origin in world             */
    double fx, fy, cx, cy;           /* pinhole                            */
    int beams, columns;              /* LiDAR                              */
    double el_max, d_el, az0, d_az;  /* radians                            */
    double near_;
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
 */
static void or_surfel_world(int i, const double* pos, const double* quat, const int* obj_id,
                            const double* obj_pose, double mu[3], double R[3][3], double Ro[3][3])
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
        for (int b = 0; b < 3; ++b) mu[a] += Ro[a][b] * pos[3 * i + b];
        for (int b = 0; b < 3; ++b) {
            R[a][b] = 0;
            for (int c = 0; c < 3; ++c) R[a][b] += Ro[a][c] * Rl[c][b];
        }
    }
}

/*
 * The composite order is an integer decision (a permutation) that rounding
 * decides: two surfels whose centre depths differ by less than FP32 can
 * resolve swap places between an FP32 and an FP64 evaluation.  The order
 * key is therefore taken in the kernel's precision -- the centre depth
 * (range) evaluated in IEEE single precision with fused multiply-adds in
 * the order the kernel uses: mu' = R_o mu + t_o, m = R mu' + t, key = m_z
 * (camera) or sqrt(m . m) (LiDAR).  Everything else stays FP64.
 */
static float or_key32(const or_sensor* S, int i, const double* pos, const int* obj_id, const double* obj_pose)
{
    float m0 = (float)pos[3 * i], m1 = (float)pos[3 * i + 1], m2 = (float)pos[3 * i + 2];
    int k = obj_id ? obj_id[i] : -1;
    if (k >= 0) {
        const double* P = obj_pose + 12 * k;
        float R[9] = {(float)P[0], (float)P[1], (float)P[2], (float)P[4], (float)P[5], (float)P[6],
                      (float)P[8], (float)P[9], (float)P[10]};
        float a0 = fmaf(R[0], m0, fmaf(R[1], m1, R[2] * m2)) + (float)P[3];
        float a1 = fmaf(R[3], m0, fmaf(R[4], m1, R[5] * m2)) + (float)P[7];
        float a2 = fmaf(R[6], m0, fmaf(R[7], m1, R[8] * m2)) + (float)P[11];
        m0 = a0; m1 = a1; m2 = a2;
    }
    float s[3];
    for (int a = 0; a < 3; ++a)
        s[a] = fmaf((float)S->Rs[a][0], m0, fmaf((float)S->Rs[a][1], m1, (float)S->Rs[a][2] * m2)) + (float)S->ts[a];
    if (S->kind == 0) return s[2];
    if (S->kind == 2) return sqrtf(fmaf(s[0], s[0], s[2] * s[2])); /* horizontal distance */
    return sqrtf(fmaf(s[0], s[0], fmaf(s[1], s[1], s[2] * s[2])));
}

static void or_prepare(or_surfel* G, int i, const or_sensor* S, const double* pos,
                       const double* log_scale, const double* quat, const double* opacity_logit,
                       int sh_degree, const double* sh, const double* intensity,
                       const double* ray_drop, const int* obj_id, const double* obj_pose)
{
    double mu[3], R[3][3], Ro[3][3];
    or_surfel_world(i, pos, quat, obj_id, obj_pose, mu, R, Ro);
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

    /* mu in the sensor frame */
    double ms[3];
    for (int a = 0; a < 3; ++a) ms[a] = S->Rs[a][0] * mu[0] + S->Rs[a][1] * mu[1] + S->Rs[a][2] * mu[2] + S->ts[a];

    G->culled = 0;
    G->key = or_key32(S, i, pos, obj_id, obj_pose);
    if (!(G->key > (float)S->near_)) { G->culled = 1; return; }  /* cull in the key's precision */
    if (S->kind == 0) {
        G->zc = ms[2];
        G->c[0] = G->WH[0][2] / G->WH[2][2];
        G->c[1] = G->WH[1][2] / G->WH[2][2];
    } else if (S->kind == 2) {
        /* cylinder: column from the azimuth about the camera's y axis, row
           from the height over the horizontal distance (pixel units) */
        G->zc = sqrt(ms[0] * ms[0] + ms[2] * ms[2]);
        G->c[0] = S->cx + S->fx * atan2(ms[0], ms[2]);
        G->c[1] = S->cy + S->fy * ms[1] / G->zc;
    } else {
        G->zc = sqrt(or_dot3(ms, ms));
        double az = atan2(ms[1], ms[0]);
        double el = atan2(ms[2], sqrt(ms[0] * ms[0] + ms[1] * ms[1]));
        /* cell coordinates: ray (row i, column j) sits at (j, i) */
        G->c[0] = (az - S->az0) / S->d_az - 0.5;
        G->c[1] = (S->el_max - el) / S->d_el;
    }
    G->o = or_sigmoid(opacity_logit[i]);

    /* normal = third column of R, in the sensor frame, facing the sensor */
    double nw[3] = {R[0][2], R[1][2], R[2][2]};
    double to_s[3] = {mu[0] - S->origin[0], mu[1] - S->origin[1], mu[2] - S->origin[2]};
    if (or_dot3(nw, to_s) > 0) { nw[0] = -nw[0]; nw[1] = -nw[1]; nw[2] = -nw[2]; }
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
                double Y = oracle_sh_basis(l, m, dl);
                for (int ch = 0; ch < 3; ++ch) col[ch] += Y * sh[((size_t)i * K + k) * 3 + ch];
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
    float key;        /* order key            */
    double zc;        /* centre depth         */
    double alpha;     /* min(0.99, o G)       */
    double z;         /* contribution depth   */
    double rho3, rholp, zint;
    int v3, vlp;      /* support validity     */
    int hasplane;     /* m2 != 0              */
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
    if (h->hasplane) {
        double u = m[0] / m[2], v = m[1] / m[2];
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
    h->vlp = h->rholp <= 9.0;
    if (!h->v3 && !h->vlp) return 0;
    double rho;
    if (h->v3 && (!h->vlp || h->rho3 <= h->rholp)) { rho = h->rho3; h->z = h->zint; }
    else { rho = h->rholp; h->z = G->zc; }
    double Gv = exp(-0.5 * rho);
    double a = G->o * Gv;
    h->alpha = a < 0.99 ? a : 0.99;
    h->zc = G->zc;
    h->key = G->key;
    return 1;
}

static int or_cmp_hit(const void* pa, const void* pb)
{
    const or_hit* a = (const or_hit*)pa;
    const or_hit* b = (const or_hit*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static double or_relm(double x, double thr) { return fabs(x - thr) / fabs(thr); }

/*
 * Decisions that FP32 rounding could flip.  A decision counts as flippable
 * when its relative distance to the threshold is below OR_FLIP_REL (2e-5),
 * and its effect is the largest
 * change of an output that flipping it could cause (T times the jump in
 * alpha; for the depth-branch choice, the relative jump in depth weight).
 */
#ifndef OR_FLIP_REL
#define OR_FLIP_REL 2e-5
#endif

typedef struct {
    double feat[3], A, B, D, N[3], T;
    double flip;      /* largest effect of a flippable decision, 0 if none */
    int n_contrib;
} or_ray;

static void or_flip(double* flip, double rel, double scale, double effect)
{
    if (rel < scale && effect > *flip) *flip = effect;
}

/*
 * Front-to-back compositing of one ray over all surfels (3DGS order and
 * thresholds), accumulating sum w feat, A = sum w, B = sum w z, D = sum w z^2
 * and sum w n, with w = alpha T.
 */
static void or_composite(const or_surfel* G, int n, const or_sensor* S, const double hu[4], const double hv[4],
                         const double d[3], const double pc[2], or_hit* buf, or_ray* out)
{
    int nh = 0;
    for (int i = 0; i < n; ++i) {
        if (G[i].culled) continue;
        or_hit h;
        h.idx = i;
        int any = or_eval(&G[i], S, hu, hv, d, pc, &h);
        /* keep near misses too: their acceptance could flip in FP32 */
        int near_miss = (h.hasplane && h.zint > S->near_ && or_relm(h.rho3, 9.0) < 1e-3) ||
                        (h.hasplane && h.rho3 <= 9.0 && or_relm(h.zint, S->near_) < 1e-3) ||
                        or_relm(h.rholp, 9.0) < 1e-3;
        if (!any && !near_miss) continue;
        if (!any) { h.alpha = 0; h.z = G[i].zc; h.zc = G[i].zc; h.key = G[i].key; }
        buf[nh++] = h;
    }
    qsort(buf, (size_t)nh, sizeof(or_hit), or_cmp_hit);
    double T = 1.0, flip = 0.0;
    double F[3] = {0, 0, 0}, A = 0, B = 0, D = 0, N[3] = {0, 0, 0};
    int nc = 0;
    for (int j = 0; j < nh; ++j) {
        const or_hit* h = &buf[j];
        const or_surfel* g = &G[h->idx];
        double edge = T * g->o * exp(-4.5);
        if (h->hasplane && h->zint > S->near_) or_flip(&flip, or_relm(h->rho3, 9.0), OR_FLIP_REL, edge);
        if (h->hasplane && h->rho3 <= 9.0)
            or_flip(&flip, or_relm(h->zint, S->near_), OR_FLIP_REL, T * g->o * exp(-0.5 * h->rho3));
        or_flip(&flip, or_relm(h->rholp, 9.0), OR_FLIP_REL, edge);
        if (h->alpha <= 0) continue;
        or_flip(&flip, or_relm(h->alpha, 1.0 / 255.0), OR_FLIP_REL, T / 255.0);
        if (h->v3 && h->vlp) {
            double big = h->rho3 > h->rholp ? h->rho3 : h->rholp;
            or_flip(&flip, fabs(h->rho3 - h->rholp) / big, OR_FLIP_REL,
                    h->alpha * T * fabs(h->zint - g->zc) / g->zc);
        }
        if (h->alpha < 1.0 / 255.0) continue;
        double test = T * (1.0 - h->alpha);
        or_flip(&flip, or_relm(test, 1e-4), OR_FLIP_REL, h->alpha * T);
        if (test < 1e-4) break;
        double w = h->alpha * T;
        for (int ch = 0; ch < 3; ++ch) F[ch] += w * g->feat[ch];
        A += w;
        B += w * h->z;
        D += w * h->z * h->z;
        for (int a = 0; a < 3; ++a) N[a] += w * g->normal[a];
        T = test;
        ++nc;
    }
    for (int ch = 0; ch < 3; ++ch) out->feat[ch] = F[ch];
    out->A = A; out->B = B; out->D = D;
    for (int a = 0; a < 3; ++a) out->N[a] = N[a];
    out->T = T;
    out->flip = flip;
    out->n_contrib = nc;
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
 * Pinhole camera frame (Eq. 3).  Pixel (x, y) has centre (x+0.5, y+0.5).
 * pix == NULL renders every pixel (n_pix = width*height, row-major), else
 * the n_pix listed pixels y*width+x.  Outputs are pixel-major:
 * rgb/normal [n_pix][3], the rest [n_pix].  rgb includes bg*T; depth is
 * sum(w z)/sum(w) (0 where sum(w) == 0); normal is sum(w n), unnormalised;
 * acc = [sum w, sum w z, sum w z^2] per pixel ([n_pix][3], may be NULL).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_render_pinhole(int n, const double* pos, const double* log_scale, const double* quat,
                          const double* opacity_logit, int sh_degree, const double* sh,
                          const int* obj_id, const double* obj_pose,
                          int width, int height, double fx, double fy, double cx, double cy,
                          double near_, const double* world_to_cam, const double* bg,
                          int n_pix, const long long* pix,
                          double* rgb, double* depth, double* normal, double* alpha, double* trans,
                          double* acc, double* flip, int* n_contrib)
{
    if (n < 0 || width <= 0 || height <= 0 || sh_degree < 0 || sh_degree > 3) return -1;
    or_sensor S;
    memset(&S, 0, sizeof(S));
    S.kind = 0;
    or_sensor_from_matrix(&S, world_to_cam);
    S.fx = fx; S.fy = fy; S.cx = cx; S.cy = cy; S.near_ = near_;
    or_surfel* G = or_prepare_all(n, &S, pos, log_scale, quat, opacity_logit, sh_degree, sh, NULL, NULL, obj_id, obj_pose);
    if (!G) return -1;
    long long npx = pix ? n_pix : (long long)width * height;
    int fail = 0;
#pragma omp parallel
    {
        or_hit* buf = (or_hit*)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (long long q = 0; q < npx; ++q) {
                long long li = pix ? pix[q] : q;
                int x = (int)(li % width), y = (int)(li / width);
                double px = x + 0.5, py = y + 0.5;
                double hu[4] = {-1, 0, 0, px}; /* Eq. 3 */
                double hv[4] = {0, -1, 0, py};
                double pc[2] = {px, py};
                double d[3] = {0, 0, 1};
                or_ray r;
                or_composite(G, n, &S, hu, hv, d, pc, buf, &r);
                for (int ch = 0; ch < 3; ++ch) rgb[q * 3 + ch] = r.feat[ch] + r.T * bg[ch];
                depth[q] = r.A > 0 ? r.B / r.A : 0.0;
                for (int a = 0; a < 3; ++a) normal[q * 3 + a] = r.N[a];
                alpha[q] = r.A;
                trans[q] = r.T;
                if (acc) { acc[q * 3 + 0] = r.A; acc[q * 3 + 1] = r.B; acc[q * 3 + 2] = r.D; }
                if (flip) flip[q] = r.flip;
                if (n_contrib) n_contrib[q] = r.n_contrib;
            }
            free(buf);
        }
    }
    free(G);
    return fail ? -1 : 0;
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
 * Outputs as oracle_render_pinhole.
 */
int oracle_render_cylindrical(int n, const double* pos, const double* log_scale, const double* quat,
                              const double* opacity_logit, int sh_degree, const double* sh,
                              const int* obj_id, const double* obj_pose,
                              int width, int height, double fx, double fy, double cx, double cy,
                              double near_, const double* world_to_cam, const double* bg,
                              int n_pix, const long long* pix,
                              double* rgb, double* depth, double* normal, double* alpha, double* trans,
                              double* acc, double* flip, int* n_contrib)
{
    if (n < 0 || width <= 0 || height <= 0 || sh_degree < 0 || sh_degree > 3) return -1;
    or_sensor S;
    memset(&S, 0, sizeof(S));
    S.kind = 2;
    or_sensor_from_matrix(&S, world_to_cam);
    S.fx = fx; S.fy = fy; S.cx = cx; S.cy = cy; S.near_ = near_;
    or_surfel* G = or_prepare_all(n, &S, pos, log_scale, quat, opacity_logit, sh_degree, sh, NULL, NULL, obj_id, obj_pose);
    if (!G) return -1;
    long long npx = pix ? n_pix : (long long)width * height;
    int fail = 0;
#pragma omp parallel
    {
        or_hit* buf = (or_hit*)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (long long q = 0; q < npx; ++q) {
                long long li = pix ? pix[q] : q;
                int x = (int)(li % width), y = (int)(li / width);
                double px = x + 0.5, py = y + 0.5;
                double phi = (px - cx) / fx, yn = (py - cy) / fy;
                double hu[4] = {cos(phi), 0, -sin(phi), 0}; /* Eq. 4 */
                double hv[4] = {yn * sin(phi), -1, yn * cos(phi), 0};
                double pc[2] = {px, py};
                double dh[3] = {sin(phi), 0, cos(phi)};   /* horizontal part of the ray */
                or_ray r;
                or_composite(G, n, &S, hu, hv, dh, pc, buf, &r);
                for (int ch = 0; ch < 3; ++ch) rgb[q * 3 + ch] = r.feat[ch] + r.T * bg[ch];
                depth[q] = r.A > 0 ? r.B / r.A : 0.0;
                for (int a = 0; a < 3; ++a) normal[q * 3 + a] = r.N[a];
                alpha[q] = r.A;
                trans[q] = r.T;
                if (acc) { acc[q * 3 + 0] = r.A; acc[q * 3 + 1] = r.B; acc[q * 3 + 2] = r.D; }
                if (flip) flip[q] = r.flip;
                if (n_contrib) n_contrib[q] = r.n_contrib;
            }
            free(buf);
        }
    }
    free(G);
    return fail ? -1 : 0;
}

/*
 * Spinning LiDAR range image (Eq. 5).  Row i (beam) has elevation
 * el_max - i (el_max - el_min)/(beams-1); column j has azimuth
 * az0 + (j+0.5) 360/columns.  Outputs per ray: range = sum(w t)/sum(w)
 * (0 where sum(w) == 0), intensity = sum(w r), acc = sum(w), T, and the
 * ray-drop probability sum(w rho) + T with rho = sigmoid(ray_drop logit)
 * of each surfel (Sec. III-A lists rho among the LiDAR scene's attributes;
 * composited like the intensity, a ray that leaves the scene returns
 * nothing).  ray_drop may be NULL (rho = 0).
 */
int oracle_render_lidar(int n, const double* pos, const double* log_scale, const double* quat,
                        const double* opacity_logit, const double* intensity, const double* ray_drop,
                        const int* obj_id, const double* obj_pose,
                        int beams, int columns, double el_min_deg, double el_max_deg, double az0_deg,
                        double near_, const double* world_to_lidar,
                        int n_ray, const long long* ray,
                        double* range, double* intens, double* drop, double* alpha, double* trans, double* flip,
                        int* n_contrib)
{
    if (n < 0 || beams < 2 || columns <= 0) return -1;
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
    int fail = 0;
#pragma omp parallel
    {
        or_hit* buf = (or_hit*)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (long long q = 0; q < nr; ++q) {
                long long li = ray ? ray[q] : q;
                int j = (int)(li % columns), i = (int)(li / columns);
                double el = S.el_max - i * S.d_el;
                double az = S.az0 + (j + 0.5) * S.d_az;
                double hu[4] = {sin(az), -cos(az), 0, 0}; /* Eq. 5 */
                double hv[4] = {sin(el) * cos(az), sin(el) * sin(az), -cos(el), 0};
                double d[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
                double pc[2] = {(double)j, (double)i};
                or_ray r;
                or_composite(G, n, &S, hu, hv, d, pc, buf, &r);
                range[q] = r.A > 0 ? r.B / r.A : 0.0;
                intens[q] = r.feat[0];
                if (drop) drop[q] = r.feat[1] + r.T;
                alpha[q] = r.A;
                trans[q] = r.T;
                if (flip) flip[q] = r.flip;
                if (n_contrib) n_contrib[q] = r.n_contrib;
            }
            free(buf);
        }
    }
    free(G);
    return fail ? -1 : 0;
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
    uvz[0] = sqrt(h.rho3); /* |(u,v)| */
    uvz[2] = h.zint;
    /* recover signed u, v from k x l again */
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
