/*
 * oracle.c -- plain FP64 CPU oracle for the cone-beam CT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or constant with the CUDA
 * library: the two are written independently from the same definitions.
 *
 * What it computes (paper: Eq. 1, "Ax = b + e", with A the ray/element
 * intersection operator; Sec. 2.1 forward projection; Sec. 2.2
 * backprojection; Sec. 2.3 regularization):
 *
 *   Frame (circular cone beam; the paper leaves the convention to TIGRE):
 *     volume vol[k][j][i] (x fastest), voxel centre
 *       X_ijk = ((i-(nx-1)/2) dx + ox, (j-(ny-1)/2) dy + oy, (k-(nz-1)/2) dz + oz)
 *     source      S   = DSO (cos t, sin t, 0)
 *     detector    D   = -(DSD-DSO) (cos t, sin t, 0)
 *     e_u = (-sin t, cos t, 0), e_v = (0, 0, 1)
 *     pixel (p,q) centre P = D + (u_p + offu) e_u + (v_q + offv) e_v,
 *       u_p = (p-(nu-1)/2) du, v_q = (q-(nv-1)/2) dv;  proj[a][q][p].
 *
 *   Interpolated forward projector (Sec. 2.1, interpolated projection):
 *     f~ = trilinear interpolant over voxel centres, zero outside
 *     (virtual zero voxels at index -1 and n).  The ray S->P is clipped to
 *     the support box [-1, n] (index space) -> [t_in, t_out], length len (mm);
 *     K = max(1, ceil(len/D - 1e-9)), D = accuracy * min(dx,dy,dz);
 *     h = len/K; samples at the midpoints t_in + (k+1/2) h;
 *     proj = h * sum_k f~(sample_k).
 *
 *   Voxel-driven backprojector (Sec. 2.2): per voxel centre X and angle,
 *     s = X.(cos t, sin t, 0), mag = DSD/(DSO - s),
 *     (u, v) = ((X.e_u) mag, X_z mag), bilinear over pixel centres with zero
 *     outside the detector, times a weight:
 *       FDK:      w = (DSO/(DSO-s))^2
 *       matched:  w = (dx dy dz)/(du dv) * l DSD^2/(DSO-s)^3,  l = |X - S|
 *                 (voxel volume over the cross-section of the ray tube of one
 *                 pixel at X, i.e. (dx dy dz)/(du dv) * L^3/(DSD l^2) with
 *                 L = l DSD/(DSO-s)).
 *
 *   Exact adjoint of the forward projector: each sample scatters
 *     h * (trilinear corner weight) * y into its 8 corner voxels.
 *
 *   Ray-voxel intersection (Siddon) projector (Sec. 2.1, the second
 *   projector TIGRE offers, the one Sec. 3.1 times): the volume is piecewise
 *   constant, voxel (i,j,k) filling the index-space box
 *   [i-1/2, i+1/2] x [j-1/2, j+1/2] x [k-1/2, k+1/2]; proj = sum over the
 *   voxels the segment S->P crosses of (intersection length, mm) x value.
 *   Written as Siddon's definition: the parameters of every crossing with a
 *   voxel boundary plane are collected, sorted, and each piece between
 *   consecutive crossings is charged to the voxel holding its midpoint.
 *   Its exact transpose scatters the same lengths.
 *
 *   TV (Sec. 2.3, gradient-descent minimisation of total variation):
 *     backward differences with replicate boundary (difference 0 at index 0),
 *     TV_eps(f) = sum sqrt(Dx^2 + Dy^2 + Dz^2 + eps); g = dTV_eps/df.
 *
 * Geometry is passed as a flat double array (see unpack()).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double DSO, DSD;
    int64_t n[3];    /* nx, ny, nz */
    double d[3];     /* dx, dy, dz (mm) */
    double o[3];     /* volume-centre offset (mm) */
    int64_t nu, nv;
    double du, dv, offu, offv;
    double accuracy; /* ray step in voxels */
} ogeo;

/* g = [DSO, DSD, nx, ny, nz, dx, dy, dz, ox, oy, oz,
 *      nu, nv, du, dv, offu, offv, accuracy] */
static void unpack(const double* g, ogeo* G)
{
    G->DSO = g[0];
    G->DSD = g[1];
    for (int a = 0; a < 3; ++a) {
        G->n[a] = (int64_t)g[2 + a];
        G->d[a] = g[5 + a];
        G->o[a] = g[8 + a];
    }
    G->nu = (int64_t)g[11];
    G->nv = (int64_t)g[12];
    G->du = g[13];
    G->dv = g[14];
    G->offu = g[15];
    G->offv = g[16];
    G->accuracy = g[17];
}

/* ---------------------------------------------------------------- volume */

static double vox(const ogeo* G, const double* vol, int64_t i, int64_t j, int64_t k)
{
    if (i < 0 || j < 0 || k < 0 || i >= G->n[0] || j >= G->n[1] || k >= G->n[2])
        return 0.0;
    return vol[(k * G->n[1] + j) * G->n[0] + i];
}

/* Trilinear interpolation at index-space point (x, y, z), zero outside. */
static double trilinear(const ogeo* G, const double* vol, double x, double y, double z)
{
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int64_t i = (int64_t)fx, j = (int64_t)fy, k = (int64_t)fz;
    double ax = x - fx, ay = y - fy, az = z - fz;
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        int bi = c & 1, bj = (c >> 1) & 1, bk = (c >> 2) & 1;
        double w = (bi ? ax : 1.0 - ax) * (bj ? ay : 1.0 - ay) * (bk ? az : 1.0 - az);
        acc += w * vox(G, vol, i + bi, j + bj, k + bk);
    }
    return acc;
}

/* ------------------------------------------------------------------- rays */

typedef struct {
    double xs[3];   /* source in index space */
    double r[3];    /* (P - S) in index space */
    double t_in, t_out;
    double len;     /* mm */
    int64_t K;
} oray;

/* Index-space coordinate of a world point along axis a. */
static double to_index(const ogeo* G, int a, double X)
{
    return (X - G->o[a]) / G->d[a] + 0.5 * (double)(G->n[a] - 1);
}

/* Build the ray from the source to pixel (p, q) at angle theta and clip it
 * to the interpolant's support.  Returns 0 if the ray misses the support. */
static int ray_setup(const ogeo* G, double theta, int64_t p, int64_t q, oray* R)
{
    double c = cos(theta), s = sin(theta);
    double S[3] = { G->DSO * c, G->DSO * s, 0.0 };
    double D[3] = { -(G->DSD - G->DSO) * c, -(G->DSD - G->DSO) * s, 0.0 };
    double eu[3] = { -s, c, 0.0 };
    double up = ((double)p - 0.5 * (double)(G->nu - 1)) * G->du + G->offu;
    double vq = ((double)q - 0.5 * (double)(G->nv - 1)) * G->dv + G->offv;
    double P[3];
    for (int a = 0; a < 3; ++a)
        P[a] = D[a] + up * eu[a] + (a == 2 ? vq : 0.0);
    double seg = 0.0;
    for (int a = 0; a < 3; ++a)
        seg += (P[a] - S[a]) * (P[a] - S[a]);
    seg = sqrt(seg);

    double t0 = 0.0, t1 = 1.0;
    for (int a = 0; a < 3; ++a) {
        R->xs[a] = to_index(G, a, S[a]);
        R->r[a] = (P[a] - S[a]) / G->d[a];
        double lo = -1.0, hi = (double)G->n[a];
        if (R->r[a] == 0.0) {
            if (!(R->xs[a] > lo && R->xs[a] < hi))
                return 0;
            continue;
        }
        double ta = (lo - R->xs[a]) / R->r[a];
        double tb = (hi - R->xs[a]) / R->r[a];
        if (ta > tb) {
            double tmp = ta;
            ta = tb;
            tb = tmp;
        }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (!(t1 > t0))
        return 0;
    R->t_in = t0;
    R->t_out = t1;
    R->len = (t1 - t0) * seg;
    double step = G->accuracy * fmin(G->d[0], fmin(G->d[1], G->d[2]));
    int64_t K = (int64_t)ceil(R->len / step - 1e-9);
    R->K = K < 1 ? 1 : K;
    return 1;
}

static double ray_integral(const ogeo* G, const double* vol, double theta, int64_t p, int64_t q,
                           int64_t* Kout)
{
    oray R;
    if (!ray_setup(G, theta, p, q, &R)) {
        if (Kout) *Kout = 0;
        return 0.0;
    }
    if (Kout) *Kout = R.K;
    double dt = (R.t_out - R.t_in) / (double)R.K;
    double acc = 0.0;
    for (int64_t k = 0; k < R.K; ++k) {
        double t = R.t_in + ((double)k + 0.5) * dt;
        acc += trilinear(G, vol, R.xs[0] + t * R.r[0], R.xs[1] + t * R.r[1], R.xs[2] + t * R.r[2]);
    }
    return acc * (R.len / (double)R.K);
}

/* Forward projection of the whole volume: proj has shape (na, nv, nu). */
void oracle_forward(const double* g, const double* angles, int64_t na, const double* vol,
                    double* proj)
{
    ogeo G;
    unpack(g, &G);
    int64_t rows = na * G.nv;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t aq = 0; aq < rows; ++aq) {
        int64_t a = aq / G.nv, q = aq % G.nv;
        for (int64_t p = 0; p < G.nu; ++p)
            proj[aq * G.nu + p] = ray_integral(&G, vol, angles[a], p, q, NULL);
    }
}

/* Forward projection of selected rays; idx holds (a, q, p) triplets. */
void oracle_forward_rays(const double* g, const double* angles, const double* vol,
                         const int64_t* idx, int64_t n, double* out)
{
    ogeo G;
    unpack(g, &G);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n; ++r)
        out[r] = ray_integral(&G, vol, angles[idx[3 * r]], idx[3 * r + 2], idx[3 * r + 1], NULL);
}

/* Total number of quadrature samples (sum of K over all rays). */
int64_t oracle_sample_count(const double* g, const double* angles, int64_t na)
{
    ogeo G;
    unpack(g, &G);
    int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 4)
    for (int64_t aq = 0; aq < na * G.nv; ++aq) {
        oray R;
        for (int64_t p = 0; p < G.nu; ++p)
            if (ray_setup(&G, angles[aq / G.nv], p, aq % G.nv, &R))
                total += R.K;
    }
    return total;
}

/* Per-ray (K, len, t_in, t_out) for selected rays, for tests of the clip. */
void oracle_ray_params(const double* g, const double* angles, const int64_t* idx, int64_t n,
                       double* out4)
{
    ogeo G;
    unpack(g, &G);
    for (int64_t r = 0; r < n; ++r) {
        oray R;
        if (ray_setup(&G, angles[idx[3 * r]], idx[3 * r + 2], idx[3 * r + 1], &R)) {
            out4[4 * r] = (double)R.K;
            out4[4 * r + 1] = R.len;
            out4[4 * r + 2] = R.t_in;
            out4[4 * r + 3] = R.t_out;
        } else {
            out4[4 * r] = 0.0;
            out4[4 * r + 1] = 0.0;
            out4[4 * r + 2] = 0.0;
            out4[4 * r + 3] = 0.0;
        }
    }
}

/* ---------------------------------------------------------- backprojection */

static double pix(const ogeo* G, const double* img, int64_t p, int64_t q)
{
    if (p < 0 || q < 0 || p >= G->nu || q >= G->nv)
        return 0.0;
    return img[q * G->nu + p];
}

/* Contribution of one angle to voxel (i, j, k); mode 0 = matched, 1 = FDK. */
static double bp_one(const ogeo* G, const double* img, double theta, int64_t i, int64_t j,
                     int64_t k, int mode)
{
    double X[3];
    int64_t ijk[3] = { i, j, k };
    for (int a = 0; a < 3; ++a)
        X[a] = ((double)ijk[a] - 0.5 * (double)(G->n[a] - 1)) * G->d[a] + G->o[a];
    double c = cos(theta), s = sin(theta);
    double sdist = X[0] * c + X[1] * s;
    double den = G->DSO - sdist;
    if (!(den > 0.0))
        return 0.0;
    double mag = G->DSD / den;
    double u = (-X[0] * s + X[1] * c) * mag;
    double v = X[2] * mag;
    double pu = (u - G->offu) / G->du + 0.5 * (double)(G->nu - 1);
    double pv = (v - G->offv) / G->dv + 0.5 * (double)(G->nv - 1);
    double fu = floor(pu), fv = floor(pv);
    int64_t p0 = (int64_t)fu, q0 = (int64_t)fv;
    double au = pu - fu, av = pv - fv;
    double val = (1.0 - au) * (1.0 - av) * pix(G, img, p0, q0) +
                 au * (1.0 - av) * pix(G, img, p0 + 1, q0) +
                 (1.0 - au) * av * pix(G, img, p0, q0 + 1) + au * av * pix(G, img, p0 + 1, q0 + 1);
    double w;
    if (mode == 1) {
        w = (G->DSO / den) * (G->DSO / den);
    } else {
        double Sx = G->DSO * c, Sy = G->DSO * s;
        double l = sqrt((X[0] - Sx) * (X[0] - Sx) + (X[1] - Sy) * (X[1] - Sy) + X[2] * X[2]);
        w = (G->d[0] * G->d[1] * G->d[2]) / (G->du * G->dv) * l * G->DSD * G->DSD /
            (den * den * den);
    }
    return w * val;
}

/* Voxel-driven backprojection of proj (na, nv, nu) into vol (nz, ny, nx). */
void oracle_backward(const double* g, const double* angles, int64_t na, const double* proj,
                     double* vol, int mode)
{
    ogeo G;
    unpack(g, &G);
    int64_t planes = G.n[2] * G.n[1];
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t kj = 0; kj < planes; ++kj) {
        int64_t k = kj / G.n[1], j = kj % G.n[1];
        for (int64_t i = 0; i < G.n[0]; ++i) {
            double acc = 0.0;
            for (int64_t a = 0; a < na; ++a)
                acc += bp_one(&G, proj + a * G.nu * G.nv, angles[a], i, j, k, mode);
            vol[kj * G.n[0] + i] = acc;
        }
    }
}

/* Backprojection at selected voxels; idx holds (i, j, k) triplets. */
void oracle_backward_voxels(const double* g, const double* angles, int64_t na, const double* proj,
                            const int64_t* idx, int64_t n, double* out, int mode)
{
    ogeo G;
    unpack(g, &G);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int64_t a = 0; a < na; ++a)
            acc += bp_one(&G, proj + a * G.nu * G.nv, angles[a], idx[3 * r], idx[3 * r + 1],
                          idx[3 * r + 2], mode);
        out[r] = acc;
    }
}

/* ---------------------------------------------------------- exact adjoint */

/* Scatter every sample of one ray into vol_out (serial within the ray). */
static void ray_scatter(const ogeo* G, double theta, int64_t p, int64_t q, double y, double* out)
{
    oray R;
    if (y == 0.0 || !ray_setup(G, theta, p, q, &R))
        return;
    double dt = (R.t_out - R.t_in) / (double)R.K;
    double h = R.len / (double)R.K;
    for (int64_t k = 0; k < R.K; ++k) {
        double t = R.t_in + ((double)k + 0.5) * dt;
        double x = R.xs[0] + t * R.r[0], yy = R.xs[1] + t * R.r[1], z = R.xs[2] + t * R.r[2];
        double fx = floor(x), fy = floor(yy), fz = floor(z);
        int64_t i = (int64_t)fx, j = (int64_t)fy, kk = (int64_t)fz;
        double ax = x - fx, ay = yy - fy, az = z - fz;
        for (int c = 0; c < 8; ++c) {
            int bi = c & 1, bj = (c >> 1) & 1, bk = (c >> 2) & 1;
            int64_t ii = i + bi, jj = j + bj, kz = kk + bk;
            if (ii < 0 || jj < 0 || kz < 0 || ii >= G->n[0] || jj >= G->n[1] || kz >= G->n[2])
                continue;
            double w = (bi ? ax : 1.0 - ax) * (bj ? ay : 1.0 - ay) * (bk ? az : 1.0 - az);
            out[(kz * G->n[1] + jj) * G->n[0] + ii] += h * w * y;
        }
    }
}

/* Exact transpose of oracle_forward: vol_out = A^T proj (serial). */
void oracle_adjoint(const double* g, const double* angles, int64_t na, const double* proj,
                    double* vol_out)
{
    ogeo G;
    unpack(g, &G);
    memset(vol_out, 0, sizeof(double) * (size_t)(G.n[0] * G.n[1] * G.n[2]));
    for (int64_t a = 0; a < na; ++a)
        for (int64_t q = 0; q < G.nv; ++q)
            for (int64_t p = 0; p < G.nu; ++p)
                ray_scatter(&G, angles[a], p, q, proj[(a * G.nv + q) * G.nu + p], vol_out);
}

/* World position of the centre of voxel index (i, j, k) (fractional allowed). */
static void index_to_world(const ogeo* G, const double* ijk, double* X)
{
    for (int a = 0; a < 3; ++a)
        X[a] = (ijk[a] - 0.5 * (double)(G->n[a] - 1)) * G->d[a] + G->o[a];
}

/* Detector pixel coordinates (fractional index) of world point X at theta. */
static void world_to_pixel(const ogeo* G, double theta, const double* X, double* pq)
{
    double c = cos(theta), s = sin(theta);
    double den = G->DSO - (X[0] * c + X[1] * s);
    double mag = G->DSD / den;
    double u = (-X[0] * s + X[1] * c) * mag, v = X[2] * mag;
    pq[0] = (u - G->offu) / G->du + 0.5 * (double)(G->nu - 1);
    pq[1] = (v - G->offv) / G->dv + 0.5 * (double)(G->nv - 1);
}

/* Exact adjoint at selected voxels.  Only rays whose samples can reach the
 * voxel's 8-neighbourhood matter: those through the box [i-1, i+1] x
 * [j-1, j+1] x [k-1, k+1]; the pixel window is the bounding box of the
 * projections of its corners, widened by one pixel. */
void oracle_adjoint_voxels(const double* g, const double* angles, int64_t na, const double* proj,
                           const int64_t* idx, int64_t n, double* out)
{
    ogeo G;
    unpack(g, &G);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n; ++r) {
        int64_t vi = idx[3 * r], vj = idx[3 * r + 1], vk = idx[3 * r + 2];
        double acc = 0.0;
        for (int64_t a = 0; a < na; ++a) {
            double pmin = 1e300, pmax = -1e300, qmin = 1e300, qmax = -1e300;
            for (int c = 0; c < 8; ++c) {
                double ijk[3] = { (double)vi + ((c & 1) ? 1.0 : -1.0),
                                  (double)vj + ((c & 2) ? 1.0 : -1.0),
                                  (double)vk + ((c & 4) ? 1.0 : -1.0) };
                double X[3], pq[2];
                index_to_world(&G, ijk, X);
                world_to_pixel(&G, angles[a], X, pq);
                pmin = fmin(pmin, pq[0]);
                pmax = fmax(pmax, pq[0]);
                qmin = fmin(qmin, pq[1]);
                qmax = fmax(qmax, pq[1]);
            }
            int64_t p0 = (int64_t)floor(pmin) - 1, p1 = (int64_t)ceil(pmax) + 1;
            int64_t q0 = (int64_t)floor(qmin) - 1, q1 = (int64_t)ceil(qmax) + 1;
            if (p0 < 0) p0 = 0;
            if (q0 < 0) q0 = 0;
            if (p1 > G.nu - 1) p1 = G.nu - 1;
            if (q1 > G.nv - 1) q1 = G.nv - 1;
            for (int64_t q = q0; q <= q1; ++q)
                for (int64_t p = p0; p <= p1; ++p) {
                    double y = proj[(a * G.nv + q) * G.nu + p];
                    oray R;
                    if (y == 0.0 || !ray_setup(&G, angles[a], p, q, &R))
                        continue;
                    double dt = (R.t_out - R.t_in) / (double)R.K;
                    double h = R.len / (double)R.K;
                    for (int64_t k = 0; k < R.K; ++k) {
                        double t = R.t_in + ((double)k + 0.5) * dt;
                        double x = R.xs[0] + t * R.r[0], yy = R.xs[1] + t * R.r[1],
                               z = R.xs[2] + t * R.r[2];
                        double ax = 1.0 - fabs(x - (double)vi);
                        double ay = 1.0 - fabs(yy - (double)vj);
                        double az = 1.0 - fabs(z - (double)vk);
                        if (ax > 0.0 && ay > 0.0 && az > 0.0)
                            acc += h * ax * ay * az * y;
                    }
                }
        }
        out[r] = acc;
    }
}

/* ----------------------------------------------------- Siddon projector */

typedef struct {
    double xs[3];  /* source, index space */
    double r[3];   /* P - S, index space */
    double seg;    /* |P - S| (mm) */
    double t0, t1; /* clip of t in [0, 1] to the voxel boxes' hull */
} sray;

/* Ray from the source to pixel (p, q), clipped to [-1/2, n-1/2] per axis
 * (the union of the voxel boxes).  Returns 0 if it misses. */
static int siddon_setup(const ogeo* G, double theta, int64_t p, int64_t q, sray* R)
{
    double c = cos(theta), s = sin(theta);
    double S[3] = { G->DSO * c, G->DSO * s, 0.0 };
    double D[3] = { -(G->DSD - G->DSO) * c, -(G->DSD - G->DSO) * s, 0.0 };
    double eu[3] = { -s, c, 0.0 };
    double up = ((double)p - 0.5 * (double)(G->nu - 1)) * G->du + G->offu;
    double vq = ((double)q - 0.5 * (double)(G->nv - 1)) * G->dv + G->offv;
    double seg = 0.0;
    R->t0 = 0.0;
    R->t1 = 1.0;
    for (int a = 0; a < 3; ++a) {
        double P = D[a] + up * eu[a] + (a == 2 ? vq : 0.0);
        seg += (P - S[a]) * (P - S[a]);
        R->xs[a] = to_index(G, a, S[a]);
        R->r[a] = (P - S[a]) / G->d[a];
    }
    R->seg = sqrt(seg);
    for (int a = 0; a < 3; ++a) {
        double lo = -0.5, hi = (double)G->n[a] - 0.5;
        if (R->r[a] == 0.0) {
            if (!(R->xs[a] > lo && R->xs[a] < hi))
                return 0;
            continue;
        }
        double ta = (lo - R->xs[a]) / R->r[a], tb = (hi - R->xs[a]) / R->r[a];
        if (ta > tb) {
            double tmp = ta;
            ta = tb;
            tb = tmp;
        }
        if (ta > R->t0) R->t0 = ta;
        if (tb < R->t1) R->t1 = tb;
    }
    return R->t1 > R->t0;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Line integral of one ray (scatter == NULL), or scatter y times the
 * intersection lengths into scatter (vol-shaped). */
static double siddon_ray(const ogeo* G, const double* vol, double theta, int64_t p, int64_t q,
                         double* scatter, double y)
{
    sray R;
    if (!siddon_setup(G, theta, p, q, &R))
        return 0.0;
    int64_t cap = 2 + (G->n[0] - 1) + (G->n[1] - 1) + (G->n[2] - 1);
    double* ts = (double*)malloc(sizeof(double) * (size_t)cap);
    int64_t m = 0;
    ts[m++] = R.t0;
    ts[m++] = R.t1;
    for (int a = 0; a < 3; ++a) {
        if (R.r[a] == 0.0)
            continue;
        for (int64_t b = 1; b < G->n[a]; ++b) {
            double t = ((double)b - 0.5 - R.xs[a]) / R.r[a];
            if (t > R.t0 && t < R.t1)
                ts[m++] = t;
        }
    }
    qsort(ts, (size_t)m, sizeof(double), cmp_double);
    double acc = 0.0;
    for (int64_t e = 0; e + 1 < m; ++e) {
        double ta = ts[e], tb = ts[e + 1];
        if (!(tb > ta))
            continue;
        double tm = 0.5 * (ta + tb);
        int64_t ijk[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            ijk[a] = (int64_t)floor(R.xs[a] + tm * R.r[a] + 0.5);
            if (ijk[a] < 0 || ijk[a] >= G->n[a])
                inside = 0;
        }
        if (!inside)
            continue;
        int64_t v = (ijk[2] * G->n[1] + ijk[1]) * G->n[0] + ijk[0];
        double L = (tb - ta) * R.seg;
        if (scatter)
            scatter[v] += L * y;
        else
            acc += L * vol[v];
    }
    free(ts);
    return acc;
}

/* Siddon forward projection of the whole volume: proj (na, nv, nu). */
void oracle_siddon_forward(const double* g, const double* angles, int64_t na, const double* vol,
                           double* proj)
{
    ogeo G;
    unpack(g, &G);
    int64_t rows = na * G.nv;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t aq = 0; aq < rows; ++aq) {
        int64_t a = aq / G.nv, q = aq % G.nv;
        for (int64_t p = 0; p < G.nu; ++p)
            proj[aq * G.nu + p] = siddon_ray(&G, vol, angles[a], p, q, NULL, 0.0);
    }
}

/* Siddon projection of selected rays; idx holds (a, q, p) triplets. */
void oracle_siddon_forward_rays(const double* g, const double* angles, const double* vol,
                                const int64_t* idx, int64_t n, double* out)
{
    ogeo G;
    unpack(g, &G);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n; ++r)
        out[r] = siddon_ray(&G, vol, angles[idx[3 * r]], idx[3 * r + 2], idx[3 * r + 1], NULL, 0.0);
}

/* Exact transpose of oracle_siddon_forward (serial scatter). */
void oracle_siddon_adjoint(const double* g, const double* angles, int64_t na, const double* proj,
                           double* vol_out)
{
    ogeo G;
    unpack(g, &G);
    memset(vol_out, 0, sizeof(double) * (size_t)(G.n[0] * G.n[1] * G.n[2]));
    for (int64_t a = 0; a < na; ++a)
        for (int64_t q = 0; q < G.nv; ++q)
            for (int64_t p = 0; p < G.nu; ++p) {
                double y = proj[(a * G.nv + q) * G.nu + p];
                if (y != 0.0)
                    siddon_ray(&G, NULL, angles[a], p, q, vol_out, y);
            }
}

/* --------------------------------------------------------------------- TV */

/* Backward differences at voxel (i, j, k); zero across the low boundary. */
static void tv_at(const double* f, int64_t nx, int64_t ny, int64_t i, int64_t j, int64_t k,
                  double* Dx, double* Dy, double* Dz)
{
    int64_t c = (k * ny + j) * nx + i;
    *Dx = i > 0 ? f[c] - f[c - 1] : 0.0;
    *Dy = j > 0 ? f[c] - f[c - nx] : 0.0;
    *Dz = k > 0 ? f[c] - f[c - nx * ny] : 0.0;
}

/* TV_eps(f) = sum over voxels of sqrt(Dx^2 + Dy^2 + Dz^2 + eps). */
double oracle_tv_value(const double* f, int64_t nx, int64_t ny, int64_t nz, double eps)
{
    double total = 0.0;
#pragma omp parallel for reduction(+ : total)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double Dx, Dy, Dz;
                tv_at(f, nx, ny, i, j, k, &Dx, &Dy, &Dz);
                total += sqrt(Dx * Dx + Dy * Dy + Dz * Dz + eps);
            }
    return total;
}

/* g = dTV_eps/df.  Voxel c appears in its own term (through +Dx, +Dy, +Dz
 * when the index is > 0) and in the terms of its forward neighbours
 * (i+1, j+1, k+1), where it enters with a minus sign. */
static double tv_grad_at(const double* f, int64_t nx, int64_t ny, int64_t nz, int64_t i,
                         int64_t j, int64_t k, double eps)
{
    double Dx, Dy, Dz, gsum = 0.0;
    tv_at(f, nx, ny, i, j, k, &Dx, &Dy, &Dz);
    gsum += (Dx + Dy + Dz) / sqrt(Dx * Dx + Dy * Dy + Dz * Dz + eps);
    if (i + 1 < nx) {
        tv_at(f, nx, ny, i + 1, j, k, &Dx, &Dy, &Dz);
        gsum -= Dx / sqrt(Dx * Dx + Dy * Dy + Dz * Dz + eps);
    }
    if (j + 1 < ny) {
        tv_at(f, nx, ny, i, j + 1, k, &Dx, &Dy, &Dz);
        gsum -= Dy / sqrt(Dx * Dx + Dy * Dy + Dz * Dz + eps);
    }
    if (k + 1 < nz) {
        tv_at(f, nx, ny, i, j, k + 1, &Dx, &Dy, &Dz);
        gsum -= Dz / sqrt(Dx * Dx + Dy * Dy + Dz * Dz + eps);
    }
    return gsum;
}

void oracle_tv_grad(const double* f, int64_t nx, int64_t ny, int64_t nz, double eps, double* g)
{
#pragma omp parallel for
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                g[(k * ny + j) * nx + i] = tv_grad_at(f, nx, ny, nz, i, j, k, eps);
}

/* Gradient at selected voxels (i, j, k) triplets. */
void oracle_tv_grad_voxels(const double* f, int64_t nx, int64_t ny, int64_t nz, double eps,
                           const int64_t* idx, int64_t n, double* out)
{
#pragma omp parallel for
    for (int64_t r = 0; r < n; ++r)
        out[r] = tv_grad_at(f, nx, ny, nz, idx[3 * r], idx[3 * r + 1], idx[3 * r + 2], eps);
}

/* n_steps of x <- x - alpha g/||g||_2 (no-op when ||g|| = 0), in place. */
void oracle_tv_steps(double* f, int64_t nx, int64_t ny, int64_t nz, int n_steps, double alpha,
                     double eps)
{
    int64_t N = nx * ny * nz;
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    for (int s = 0; s < n_steps; ++s) {
        oracle_tv_grad(f, nx, ny, nz, eps, g);
        double nn = 0.0;
        for (int64_t c = 0; c < N; ++c)
            nn += g[c] * g[c];
        nn = sqrt(nn);
        if (nn == 0.0)
            continue;
        for (int64_t c = 0; c < N; ++c)
            f[c] -= alpha * g[c] / nn;
    }
    free(g);
}
