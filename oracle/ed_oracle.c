/*
 * ed_oracle.c -- plain FP64 CPU oracle of the embedded-deformation (ED)
 * registration hot path of MIS-SLAM (Song et al., arXiv 1803.02009).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and must never be used as a fallback for it.
 *
 * Every function restates a step of the paper in its order and notation, in
 * double precision, with no blocking or fusion:
 *   Sec. II.D  Eq. (1) warp, Eq. (2) skinning weight, node sampling
 *   Sec. II.E  Eq. (3) energy: E_rot, E_reg, E_data (+ visibility gate),
 *              E_r / E_p pose priors, E_corr key correspondences
 *   Sec. II.F  Levenberg-Marquardt / Gauss-Newton step
 *   Sec. II.G  Algorithm 1 (point-to-depth registration), Algorithm 2
 *              (deform, register, fuse, lift, delete), fusion Eqs. (fusion1-4),
 *              Algorithm 3 (box downsampling, Sec. III.A)
 *   Sec. III   back-projection error (projected model image - depth image)
 *
 * Integer decisions (projection to a pixel, nearest-node keys, the
 * visibility / registration gates, the z-buffer) are taken in FP32 by the
 * exact operation orders below, so that they are bit-identical to any other
 * implementation that follows the same rule on the same float inputs.  Build
 * with -ffp-contract=off (no fused multiply-add) on an SSE target.
 *
 * Readings of passages the paper leaves open (each one also applies to any
 * implementation checked against this oracle):
 *   weights are normalised to sum to one (Eq. 1 has no normalisation);
 *   P(v) rounds x/z*fx+cx to the nearest pixel centre (floor(t + 0.5));
 *   nearest nodes use the FP32 squared distance, ties to the lower index;
 *   nodes come from a phase-ordered Poisson-disk sampler (27 phases);
 *   the node graph N(j) is the KG nearest other nodes, alpha_jk = 1;
 *   the normal gate is angle < eps_n, i.e. dot > cos(eps_n);
 *   all energy terms are squared (least squares);
 *   the pose is (alpha, beta, gamma, T), R = Rz(gamma) Ry(beta) Rx(alpha);
 *   the observation weight in the fusion equations is 1, the TSDW formula
 *   only acts as the |z - D| < tau gate; omega_max is a parameter (20).
 *
 * The oracle is this file compiled without OpenMP.  The same source compiled
 * with -fopenmp (liboracle_omp.so) is only timed, as the multi-core CPU
 * baseline: its per-point and per-node loops run in parallel (each iteration
 * writes its own outputs), the sort of the block pattern runs as per-thread
 * sorts and a merge (the same result), and the data term of the normal
 * equations is summed per thread over contiguous point ranges, the thread
 * sums then added in thread order (a fixed order, so the result is
 * deterministic for a given thread count, and equal to the oracle's up to
 * rounding).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_CAPACITY 3
#define OR_ERR_BREAKDOWN 5
#define OR_MAXK 64   /* largest K of the nearest-node searches */

/* ------------------------------------------------------------------------- */
/* FP32 decision rules (bit-exact)                                            */
/* ------------------------------------------------------------------------- */

/* squared distance key: dx*dx + dy*dy + dz*dz, left to right, no FMA */
static float key_f32(float px, float py, float pz, float gx, float gy, float gz)
{
    float dx = px - gx;
    float dy = py - gy;
    float dz = pz - gz;
    float s = dx * dx;
    float t = dy * dy;
    s = s + t;
    t = dz * dz;
    s = s + t;
    return s;
}

/* P(v): pixel of a camera-frame point.  q = x/z, t = fx*q, t = t + cx,
 * t = t + 0.5, u = floor(t); same for v.  Returns 0 when off image. */
static int project_f32(float x, float y, float z, float fx, float fy, float cx, float cy,
                       int W, int H, int *pu, int *pv)
{
    if (!(z > 0.0f))
        return 0;
    float qx = x / z;
    float tx = fx * qx;
    tx = tx + cx;
    tx = tx + 0.5f;
    float qy = y / z;
    float ty = fy * qy;
    ty = ty + cy;
    ty = ty + 0.5f;
    float fu = floorf(tx), fv = floorf(ty);
    if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H))
        return 0;
    *pu = (int)fu;
    *pv = (int)fv;
    return 1;
}

/* Pi(u, D) in FP32 for the gates: ((u - cx) * D / fx, (v - cy) * D / fy, D) */
static void backproject_f32(int u, int v, float D, float fx, float fy, float cx, float cy, float *out)
{
    float a = (float)u - cx;
    a = a * D;
    a = a / fx;
    float b = (float)v - cy;
    b = b * D;
    b = b / fy;
    out[0] = a;
    out[1] = b;
    out[2] = D;
}

static float dot3_f32(const float *a, const float *b)
{
    float s = a[0] * b[0];
    float t = a[1] * b[1];
    s = s + t;
    t = a[2] * b[2];
    s = s + t;
    return s;
}

/*
 * Visible-point extraction / projective association (Sec. II.E, data term
 * gate): pixel u = P(v~); valid iff u on image, D(u) > 0, target normal
 * valid, ||v~ - Gamma(u)||^2 < eps_d^2 and n~ . n(u) > cos(eps_n), all in
 * FP32 on the given float inputs.  pix[i] = v*W + u or -1.
 */
void or_associate_f32(const float *wpos, const float *wnrm, int N, const float *depth,
                      const float *nmap, float fx, float fy, float cx, float cy, int W, int H,
                      float eps_d, float cos_eps_n, int *pix)
{
    float eps2 = eps_d * eps_d;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        const float *p = wpos + 4 * (size_t)i;
        const float *n = wnrm + 4 * (size_t)i;
        int u, v;
        pix[i] = -1;
        if (!project_f32(p[0], p[1], p[2], fx, fy, cx, cy, W, H, &u, &v))
            continue;
        size_t q = (size_t)v * W + u;
        float D = depth[q];
        if (!(D > 0.0f))
            continue;
        const float *tn = nmap + 4 * q;
        if (tn[3] == 0.0f)
            continue;
        float G[3];
        backproject_f32(u, v, D, fx, fy, cx, cy, G);
        float d[3] = {p[0] - G[0], p[1] - G[1], p[2] - G[2]};
        float d2 = dot3_f32(d, d);
        if (!(d2 < eps2))
            continue;
        float c = dot3_f32(n, tn);
        if (!(c > cos_eps_n))
            continue;
        pix[i] = (int)q;
    }
}

/* ------------------------------------------------------------------------- */
/* Target normal map (the n(u) of the data term, Sec. II.E)                   */
/* ------------------------------------------------------------------------- */

/*
 * n(u,v) = normalize( (V(u,v+h) - V(u,v-h)) x (V(u+h,v) - V(u-h,v)) ),
 * V = back-projection of the depth map, oriented so that n_z < 0 (towards the
 * camera).  Invalid (all zero) when the centre or any stencil sample is a
 * hole or off image.  FP64 arithmetic, FP32 output.
 */
void or_normals(const float *depth, int W, int H, double fx, double fy, double cx, double cy,
                int h, float *nmap)
{
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            float *o = nmap + 4 * ((size_t)v * W + u);
            o[0] = o[1] = o[2] = o[3] = 0.0f;
            if (u - h < 0 || u + h >= W || v - h < 0 || v + h >= H)
                continue;
            double Dc = depth[(size_t)v * W + u];
            double Dl = depth[(size_t)v * W + (u - h)], Dr = depth[(size_t)v * W + (u + h)];
            double Du = depth[(size_t)(v - h) * W + u], Dd = depth[(size_t)(v + h) * W + u];
            if (!(Dc > 0 && Dl > 0 && Dr > 0 && Du > 0 && Dd > 0))
                continue;
            double Vl[3] = {((u - h) - cx) * Dl / fx, (v - cy) * Dl / fy, Dl};
            double Vr[3] = {((u + h) - cx) * Dr / fx, (v - cy) * Dr / fy, Dr};
            double Vu[3] = {(u - cx) * Du / fx, ((v - h) - cy) * Du / fy, Du};
            double Vd[3] = {(u - cx) * Dd / fx, ((v + h) - cy) * Dd / fy, Dd};
            double a[3] = {Vd[0] - Vu[0], Vd[1] - Vu[1], Vd[2] - Vu[2]};
            double b[3] = {Vr[0] - Vl[0], Vr[1] - Vl[1], Vr[2] - Vl[2]};
            double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (!(len > 0))
                continue;
            double s = (n[2] > 0 ? -1.0 : 1.0) / len;
            o[0] = (float)(n[0] * s);
            o[1] = (float)(n[1] * s);
            o[2] = (float)(n[2] * s);
            o[3] = 1.0f;
        }
}

/* ------------------------------------------------------------------------- */
/* ED node sampling (Sec. II.D: nodes "sparsely and evenly scattered")        */
/* ------------------------------------------------------------------------- */

/*
 * Phase-ordered Poisson-disk sampling with radius r.  Cells of edge
 * cs = r * (1/sqrt 3) cover the points' bounding box; the 27 phases
 * (cx mod 3) + 3 (cy mod 3) + 9 (cz mod 3) are visited in increasing order,
 * the cells of one phase in increasing linear index cx + nx (cy + ny cz).
 * In each cell the lowest-index point whose FP32 key to every node chosen so
 * far is >= r*r becomes a node.  Two cells of one phase are more than r
 * apart, so the choice in one cell never depends on another cell of the same
 * phase.  Nodes are numbered in selection order; the first max_nodes are
 * returned (node_pt[] = point index), the full count in *m_total.
 * Returns OR_ERR_CAPACITY when the grid would exceed max_cells.
 */
int or_poisson_nodes(const float *pos, int N, float r, int max_nodes, long max_cells, int *node_pt,
                     int *m_total)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            float c = pos[4 * (size_t)i + d];
            if (c < mn[d]) mn[d] = c;
            if (c > mx[d]) mx[d] = c;
        }
    float cs = r * 0.577350269f;
    float inv = 1.0f / cs;
    int dim[3];
    for (int d = 0; d < 3; ++d) {
        float t = mx[d] - mn[d];
        t = t * inv;
        dim[d] = (int)floorf(t) + 1;
    }
    long ncell = (long)dim[0] * dim[1] * dim[2];
    if (ncell > max_cells || ncell <= 0)
        return OR_ERR_CAPACITY;
    int *cell_of = (int *)malloc(sizeof(int) * (size_t)N);
    int *start = (int *)calloc((size_t)ncell + 1, sizeof(int));
    int *order = (int *)malloc(sizeof(int) * (size_t)N);
    int *cell_node = (int *)malloc(sizeof(int) * (size_t)ncell);
    int *nodes = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    for (long c = 0; c < ncell; ++c)
        cell_node[c] = -1;
    for (int i = 0; i < N; ++i) {
        int c3[3];
        for (int d = 0; d < 3; ++d) {
            float t = pos[4 * (size_t)i + d] - mn[d];
            t = t * inv;
            int c = (int)floorf(t);
            if (c < 0) c = 0;
            if (c >= dim[d]) c = dim[d] - 1;
            c3[d] = c;
        }
        cell_of[i] = c3[0] + dim[0] * (c3[1] + dim[1] * c3[2]);
        start[cell_of[i] + 1]++;
    }
    for (long c = 0; c < ncell; ++c)
        start[c + 1] += start[c];
    {
        int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
        memcpy(fill, start, sizeof(int) * (size_t)ncell);
        for (int i = 0; i < N; ++i) /* increasing point index inside each cell */
            order[fill[cell_of[i]]++] = i;
        free(fill);
    }
    float r2 = r * r;
    int m = 0;
    for (int ph = 0; ph < 27; ++ph) {
        int px = ph % 3, py = (ph / 3) % 3, pz = ph / 9;
        for (long c = 0; c < ncell; ++c) {
            int cx = (int)(c % dim[0]), cy = (int)((c / dim[0]) % dim[1]), cz = (int)(c / ((long)dim[0] * dim[1]));
            if (cx % 3 != px || cy % 3 != py || cz % 3 != pz)
                continue;
            for (int s = start[c]; s < start[c + 1]; ++s) {
                int i = order[s];
                const float *p = pos + 4 * (size_t)i;
                int ok = 1;
                for (int dz = -2; dz <= 2 && ok; ++dz)
                    for (int dy = -2; dy <= 2 && ok; ++dy)
                        for (int dx = -2; dx <= 2 && ok; ++dx) {
                            int ax = cx + dx, ay = cy + dy, az = cz + dz;
                            if (ax < 0 || ay < 0 || az < 0 || ax >= dim[0] || ay >= dim[1] || az >= dim[2])
                                continue;
                            int nd = cell_node[ax + dim[0] * ((long)ay + (long)dim[1] * az)];
                            if (nd < 0)
                                continue;
                            const float *q = pos + 4 * (size_t)nodes[nd];
                            if (key_f32(p[0], p[1], p[2], q[0], q[1], q[2]) < r2)
                                ok = 0;
                        }
                if (ok) {
                    cell_node[c] = m;
                    nodes[m++] = i;
                    break;
                }
            }
        }
    }
    *m_total = m;
    for (int j = 0; j < m && j < max_nodes; ++j)
        node_pt[j] = nodes[j];
    free(cell_of);
    free(start);
    free(order);
    free(cell_node);
    free(nodes);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* k nearest nodes (Sec. II.D) and node graph N(j) (Sec. II.E, E_reg)         */
/* ------------------------------------------------------------------------- */

/* insert (key, id) into a sorted list of length len <= cap; ties -> lower id */
static void topk_insert(float *keys, int *ids, int *len, int cap, float key, int id)
{
    int n = *len;
    if (n == cap) {
        float lk = keys[n - 1];
        if (key > lk || (key == lk && id > ids[n - 1]))
            return;
        n--;
    }
    int p = n;
    while (p > 0 && (keys[p - 1] > key || (keys[p - 1] == key && ids[p - 1] > id))) {
        keys[p] = keys[p - 1];
        ids[p] = ids[p - 1];
        p--;
    }
    keys[p] = key;
    ids[p] = id;
    *len = n + 1;
}

/*
 * For each listed point (all points when sel == NULL), the K nearest nodes by
 * brute force over every node with the FP32 key; ties to the lower index.
 * idx[i*K + s], key[i*K + s] for s = 0..K-1 in increasing key order.
 */
void or_knn(const float *pos, int N, const int *sel, int nsel, const float *g, int m, int K, int *idx,
            float *key)
{
    int cnt = sel ? nsel : N;
    if (K < 1 || K > OR_MAXK)
        return;
#pragma omp parallel for schedule(dynamic, 256)
    for (int t = 0; t < cnt; ++t) {
        float kk[OR_MAXK];
        int ii[OR_MAXK];
        int i = sel ? sel[t] : t;
        const float *p = pos + 4 * (size_t)i;
        int len = 0;
        for (int j = 0; j < m; ++j)
            topk_insert(kk, ii, &len, K, key_f32(p[0], p[1], p[2], g[4 * j], g[4 * j + 1], g[4 * j + 2]), j);
        for (int s = 0; s < K; ++s) {
            idx[(size_t)t * K + s] = s < len ? ii[s] : -1;
            key[(size_t)t * K + s] = s < len ? kk[s] : INFINITY;
        }
    }
}

/* N(j): the KG nearest other nodes (FP32 key, ties to the lower index) */
void or_node_graph(const float *g, int m, int KG, int *nbr)
{
    if (KG < 1 || KG > OR_MAXK)
        return;
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < m; ++j) {
        float kk[OR_MAXK];
        int ii[OR_MAXK];
        int len = 0;
        for (int l = 0; l < m; ++l) {
            if (l == j)
                continue;
            topk_insert(kk, ii, &len, KG,
                        key_f32(g[4 * j], g[4 * j + 1], g[4 * j + 2], g[4 * l], g[4 * l + 1], g[4 * l + 2]), l);
        }
        for (int s = 0; s < KG; ++s)
            nbr[(size_t)j * KG + s] = s < len ? ii[s] : -1;
    }
}

/*
 * Skinning weights, normalised (Eq. 1 / Eq. 2).  d_s = ||v - g_{idx_s}|| in
 * FP64.  mode 0 (Gaussian): w~ = exp(-d^2 / (2 sigma^2)); mode 1 (Eq. 2):
 * w~ = 1 - d_s / d_max with d_max the distance to the (K+1)-th nearest node
 * (idx holds K+1 entries per point).  w = w~ / sum(w~); 1/K if the sum is 0.
 */
void or_skin_weights(const float *pos, int N, const float *g, const int *idx, int K, int mode,
                     double sigma, double *w)
{
    int stride = K + 1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        const float *p = pos + 4 * (size_t)i;
        double d[64];
        for (int s = 0; s < stride && s < 64; ++s) {
            int j = idx[(size_t)i * stride + s];
            if (j < 0) { d[s] = INFINITY; continue; }
            double dx = (double)p[0] - g[4 * j], dy = (double)p[1] - g[4 * j + 1], dz = (double)p[2] - g[4 * j + 2];
            d[s] = sqrt(dx * dx + dy * dy + dz * dz);
        }
        double sum = 0.0;
        double *wi = w + (size_t)i * K;
        for (int s = 0; s < K; ++s) {
            double t;
            if (mode == 0)
                t = exp(-d[s] * d[s] / (2.0 * sigma * sigma));
            else
                t = d[K] > 0.0 ? 1.0 - d[s] / d[K] : 1.0;
            if (!(t > 0.0)) t = 0.0;
            wi[s] = t;
            sum += t;
        }
        for (int s = 0; s < K; ++s)
            wi[s] = sum > 0.0 ? wi[s] / sum : 1.0 / K;
    }
}

/* ------------------------------------------------------------------------- */
/* Global pose: R = Rz(gamma) Ry(beta) Rx(alpha) and its partial derivatives  */
/* ------------------------------------------------------------------------- */

static void mat3_mul(const double *a, const double *b, double *c)
{
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            t[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
    memcpy(c, t, sizeof(t));
}

/* R and dR/dalpha, dR/dbeta, dR/dgamma (row-major 3x3 each) */
void or_rotation(const double *pose, double *R, double *dR)
{
    double ca = cos(pose[0]), sa = sin(pose[0]);
    double cb = cos(pose[1]), sb = sin(pose[1]);
    double cg = cos(pose[2]), sg = sin(pose[2]);
    double Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca}, dRx[9] = {0, 0, 0, 0, -sa, -ca, 0, ca, -sa};
    double Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb}, dRy[9] = {-sb, 0, cb, 0, 0, 0, -cb, 0, -sb};
    double Rz[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1}, dRz[9] = {-sg, -cg, 0, cg, -sg, 0, 0, 0, 0};
    double t[9];
    mat3_mul(Rz, Ry, t);
    mat3_mul(t, Rx, R);
    if (dR) {
        mat3_mul(t, dRx, dR);          /* Rz Ry dRx */
        mat3_mul(Rz, dRy, t);
        mat3_mul(t, Rx, dR + 9);       /* Rz dRy Rx */
        mat3_mul(dRz, Ry, t);
        mat3_mul(t, Rx, dR + 18);      /* dRz Ry Rx */
    }
}

static void mat3_vec(const double *M, const double *v, double *o)
{
    o[0] = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    o[1] = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    o[2] = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
}

/* ------------------------------------------------------------------------- */
/* Problem description                                                        */
/* ------------------------------------------------------------------------- */

/* Node parameters x_j: the 3x4 affine [A_j | t_j] row-major,
 * x[12 j + 4 r + c] = A_j[r][c] (c < 3), x[12 j + 4 r + 3] = t_j[r].
 * Pose: (alpha, beta, gamma, Tx, Ty, Tz).  Unknown vector: 12 m node
 * parameters followed by the 6 pose parameters. */
typedef struct {
    int N, m, K, KG;
    const double *pos;   /* N x 4 model points (w lane unused here) */
    const double *nrm;   /* N x 4 model normals */
    const int *idx;      /* N x K skinning nodes */
    const double *w;     /* N x K normalised skinning weights */
    const double *g;     /* m x 4 node positions */
    const int *nbr;      /* m x KG node graph */
    const float *depth;  /* H x W target depth (mm, 0 = hole) */
    const float *nmap;   /* H x W x 4 target normals (w = valid) */
    double fx, fy, cx, cy;
    int W, H;
    double w_data, w_rot, w_reg, w_r, w_p;
    float eps_d, cos_eps_n;
    double prior[6];
    /* sparse key correspondences (E_corr): NK model key points with their own
       skinning and 3D targets in the camera frame; weight w_corr */
    int NK;
    const double *kp_pos;  /* NK x 4 */
    const int *kp_idx;     /* NK x K */
    const double *kp_w;    /* NK x K */
    const double *kp_tgt;  /* NK x 3 */
    double w_corr;
} or_problem;

/*
 * Eq. (1): v~ = R sum_j w_j [A_j (v - g_j) + g_j + t_j] + T, and the warped
 * normal n~ = normalize(R sum_j w_j A_j n) (used by the normal gate).  Also
 * returns s = the bracketed sum (the point before the global pose).
 */
void or_warp(const or_problem *P, const double *x, const double *pose, double *wpos, double *wnrm,
             double *spre)
{
    double R[9];
    or_rotation(pose, R, NULL);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->N; ++i) {
        const double *v = P->pos + 4 * (size_t)i, *n = P->nrm + 4 * (size_t)i;
        double s[3] = {0, 0, 0}, sn[3] = {0, 0, 0};
        for (int k = 0; k < P->K; ++k) {
            int j = P->idx[(size_t)i * P->K + k];
            double wj = P->w[(size_t)i * P->K + k];
            const double *gj = P->g + 4 * (size_t)j, *xj = x + 12 * (size_t)j;
            double d[3] = {v[0] - gj[0], v[1] - gj[1], v[2] - gj[2]};
            for (int r = 0; r < 3; ++r) {
                const double *row = xj + 4 * r;
                s[r] += wj * (row[0] * d[0] + row[1] * d[1] + row[2] * d[2] + gj[r] + row[3]);
                sn[r] += wj * (row[0] * n[0] + row[1] * n[1] + row[2] * n[2]);
            }
        }
        double o[3], on[3];
        mat3_vec(R, s, o);
        mat3_vec(R, sn, on);
        double len = sqrt(on[0] * on[0] + on[1] * on[1] + on[2] * on[2]);
        for (int r = 0; r < 3; ++r) {
            wpos[3 * (size_t)i + r] = o[r] + pose[3 + r];
            if (wnrm) wnrm[3 * (size_t)i + r] = len > 0 ? on[r] / len : 0.0;
            if (spre) spre[3 * (size_t)i + r] = s[r];
        }
    }
}

/* Eq. (1) for key point k: warped position and the pre-pose sum s */
static void warp_keypoint(const or_problem *P, const double *x, const double *R, const double *pose, int k,
                          double *out, double *s)
{
    const double *v = P->kp_pos + 4 * (size_t)k;
    s[0] = s[1] = s[2] = 0.0;
    for (int q = 0; q < P->K; ++q) {
        int j = P->kp_idx[(size_t)k * P->K + q];
        double wj = P->kp_w[(size_t)k * P->K + q];
        const double *gj = P->g + 4 * (size_t)j, *xj = x + 12 * (size_t)j;
        double d[3] = {v[0] - gj[0], v[1] - gj[1], v[2] - gj[2]};
        for (int r = 0; r < 3; ++r) {
            const double *row = xj + 4 * r;
            s[r] += wj * (row[0] * d[0] + row[1] * d[1] + row[2] * d[2] + gj[r] + row[3]);
        }
    }
    mat3_vec(R, s, out);
    for (int r = 0; r < 3; ++r) out[r] += pose[3 + r];
}

/* association of the FP64 warp: the FP32 rule applied to the rounded warp */
static void associate_from_f64(const or_problem *P, const double *wpos, const double *wnrm, int *pix)
{
    float *fp = (float *)malloc(sizeof(float) * 4 * (size_t)(P->N > 0 ? P->N : 1));
    float *fn = (float *)malloc(sizeof(float) * 4 * (size_t)(P->N > 0 ? P->N : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->N; ++i)
        for (int r = 0; r < 4; ++r) {
            fp[4 * (size_t)i + r] = r < 3 ? (float)wpos[3 * (size_t)i + r] : 0.0f;
            fn[4 * (size_t)i + r] = r < 3 ? (float)wnrm[3 * (size_t)i + r] : 0.0f;
        }
    or_associate_f32(fp, fn, P->N, P->depth, P->nmap, (float)P->fx, (float)P->fy, (float)P->cx,
                     (float)P->cy, P->W, P->H, P->eps_d, P->cos_eps_n, pix);
    free(fp);
    free(fn);
}

/* ------------------------------------------------------------------------- */
/* Residuals and their Jacobian rows (Sec. II.E)                              */
/* ------------------------------------------------------------------------- */

/* Rot(A) residuals on the columns c_a of A and d rho / d x_j (6 x 12) */
static void rot_residuals(const double *xj, double *rho, double *J)
{
    double A[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            A[r][c] = xj[4 * r + c];
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {1, 2, 2, 0, 1, 2};
    for (int q = 0; q < 6; ++q) {
        int a = pa[q], b = pb[q];
        double dot = A[0][a] * A[0][b] + A[1][a] * A[1][b] + A[2][a] * A[2][b];
        rho[q] = (a == b) ? dot - 1.0 : dot;
        if (J) {
            double *row = J + 12 * q;
            memset(row, 0, sizeof(double) * 12);
            for (int r = 0; r < 3; ++r) {
                row[4 * r + a] += A[r][b];
                row[4 * r + b] += A[r][a];
            }
        }
    }
}

/* E_reg residual of edge j->k: A_j (g_k - g_j) + g_j + t_j - (g_k + t_k) */
static void reg_residual(const double *xj, const double *xk, const double *gj, const double *gk, double *e)
{
    double h[3] = {gk[0] - gj[0], gk[1] - gj[1], gk[2] - gj[2]};
    for (int r = 0; r < 3; ++r) {
        const double *row = xj + 4 * r;
        e[r] = row[0] * h[0] + row[1] * h[1] + row[2] * h[2] + gj[r] + row[3] - gk[r] - xk[4 * r + 3];
    }
}

/* data residual r = n(u)^T (v~ - Pi(u, D(u))) in FP64 */
static double data_residual(const or_problem *P, int q, const double *vt, double *nt_out)
{
    int u = q % P->W, v = q / P->W;
    double D = P->depth[q];
    double G[3] = {(u - P->cx) * D / P->fx, (v - P->cy) * D / P->fy, D};
    const float *tn = P->nmap + 4 * (size_t)q;
    double nt[3] = {tn[0], tn[1], tn[2]};
    if (nt_out) memcpy(nt_out, nt, sizeof(nt));
    return nt[0] * (vt[0] - G[0]) + nt[1] * (vt[1] - G[1]) + nt[2] * (vt[2] - G[2]);
}

/* ------------------------------------------------------------------------- */
/* Normal equations: block-sparse J^T J and J^T r                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int m;
    int nnzb;
    int *row_ptr;    /* m + 1, full symmetric pattern incl. the diagonal */
    int *col;        /* nnzb, increasing inside each row */
    double *blk;     /* nnzb x 144 (row-major 12 x 12) */
    double *C;       /* m x 72: pose-node blocks d(pose) x d(x_j), row-major 6 x 12 */
    double Hpp[36];  /* pose block */
    double *g;       /* 12 m + 6: J^T r */
    double E[6];     /* data, rot, reg, rot-prior, pos-prior, correspondence energies */
    int n_valid;
} or_normal_eq;

static int cmp_pair(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : x > y;
}

#ifdef _OPENMP
/* the same ascending order as qsort: per-thread sorts of contiguous chunks,
   then rounds of pairwise merges (OpenMP build only) */
static void sort_pairs_parallel(int64_t *a, size_t n)
{
    int T = omp_get_max_threads();
    if (T < 2 || n < 65536) {
        qsort(a, n, sizeof(int64_t), cmp_pair);
        return;
    }
    size_t *cut = (size_t *)malloc(sizeof(size_t) * (size_t)(T + 1));
    for (int t = 0; t <= T; ++t) cut[t] = n * (size_t)t / (size_t)T;
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < T; ++t) qsort(a + cut[t], cut[t + 1] - cut[t], sizeof(int64_t), cmp_pair);
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * n);
    int64_t *src = a, *dst = tmp;
    for (int w = 1; w < T; w *= 2) {
#pragma omp parallel for schedule(static, 1)
        for (int t = 0; t < T; t += 2 * w) {
            size_t lo = cut[t], mid = cut[t + w < T ? t + w : T], hi = cut[t + 2 * w < T ? t + 2 * w : T];
            size_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) dst[k++] = src[j] < src[i] ? src[j++] : src[i++];
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        int64_t *x = src; src = dst; dst = x;
    }
    if (src != a) memcpy(a, src, sizeof(int64_t) * n);
    free(tmp);
    free(cut);
}
#endif

/* sparsity pattern: node pairs sharing a point, node-graph edges, diagonal */
static void pattern_build(const or_problem *P, or_normal_eq *Q)
{
    int m = P->m, K = P->K;
    size_t cap = (size_t)(P->N + P->NK) * K * K + (size_t)m * (2 * P->KG + 1);
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (cap > 0 ? cap : 1));
    const size_t KK = (size_t)K * K;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->N; ++i)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b)
                pr[(size_t)i * KK + (size_t)a * K + b] =
                    (int64_t)P->idx[(size_t)i * K + a] * m + P->idx[(size_t)i * K + b];
    size_t n = (size_t)P->N * KK;
    for (int i = 0; i < P->NK; ++i)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b)
                pr[n++] = (int64_t)P->kp_idx[(size_t)i * K + a] * m + P->kp_idx[(size_t)i * K + b];
    for (int j = 0; j < m; ++j) {
        pr[n++] = (int64_t)j * m + j;
        for (int s = 0; s < P->KG; ++s) {
            int k = P->nbr[(size_t)j * P->KG + s];
            if (k < 0) continue;
            pr[n++] = (int64_t)j * m + k;
            pr[n++] = (int64_t)k * m + j;
        }
    }
#ifdef _OPENMP
    sort_pairs_parallel(pr, n);
#else
    qsort(pr, n, sizeof(int64_t), cmp_pair);
#endif
    size_t u = 0;
    for (size_t t = 0; t < n; ++t)
        if (u == 0 || pr[t] != pr[u - 1])
            pr[u++] = pr[t];
    Q->m = m;
    Q->nnzb = (int)u;
    Q->row_ptr = (int *)calloc((size_t)m + 1, sizeof(int));
    Q->col = (int *)malloc(sizeof(int) * (u > 0 ? u : 1));
    for (size_t t = 0; t < u; ++t) {
        Q->row_ptr[pr[t] / m + 1]++;
        Q->col[t] = (int)(pr[t] % m);
    }
    for (int j = 0; j < m; ++j)
        Q->row_ptr[j + 1] += Q->row_ptr[j];
    Q->blk = (double *)calloc(u * 144 + 1, sizeof(double));
    Q->C = (double *)calloc((size_t)m * 72 + 1, sizeof(double));
    Q->g = (double *)calloc((size_t)12 * m + 6, sizeof(double));
    memset(Q->Hpp, 0, sizeof(Q->Hpp));
    memset(Q->E, 0, sizeof(Q->E));
    Q->n_valid = 0;
}

static double *block_at(or_normal_eq *Q, int j, int l)
{
    int lo = Q->row_ptr[j], hi = Q->row_ptr[j + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (Q->col[mid] == l) return Q->blk + 144 * (size_t)mid;
        if (Q->col[mid] < l) lo = mid + 1; else hi = mid - 1;
    }
    return NULL;
}

void or_normal_eq_free(or_normal_eq *Q)
{
    free(Q->row_ptr);
    free(Q->col);
    free(Q->blk);
    free(Q->C);
    free(Q->g);
    memset(Q, 0, sizeof(*Q));
}

/* add a (J_a)^T (J_b) style outer product: blk[12x12] += s * a b^T */
static void outer12(double *blk, const double *a, const double *b, double s)
{
    for (int p = 0; p < 12; ++p)
        for (int q = 0; q < 12; ++q)
            blk[12 * p + q] += s * a[p] * b[q];
}

/*
 * One point-to-plane residual r = sw n^T (v~ - target) of a point v with
 * skinning (idx, w) and pre-pose sum s: its rows of J (w.r.t. [A_j | t_j] of
 * its nodes and the pose) added to H = J^T J, g = J^T r, C and the pose block.
 */
static void add_plane_residual(or_normal_eq *Q, const or_problem *P, const double *R, const double *dR, double r,
                               double sw, const double *nt, const double *v, const int *idx, const double *w,
                               const double *s)
{
    const int K = P->K, m = P->m;
    double a[8][12];
    double nb[3] = {R[0] * nt[0] + R[3] * nt[1] + R[6] * nt[2], R[1] * nt[0] + R[4] * nt[1] + R[7] * nt[2],
                    R[2] * nt[0] + R[5] * nt[1] + R[8] * nt[2]}; /* R^T n */
    for (int k = 0; k < K; ++k) {
        int j = idx[k];
        double wj = w[k];
        const double *gj = P->g + 4 * (size_t)j;
        double dh[4] = {v[0] - gj[0], v[1] - gj[1], v[2] - gj[2], 1.0};
        for (int rr = 0; rr < 3; ++rr)
            for (int c = 0; c < 4; ++c)
                a[k][4 * rr + c] = sw * wj * nb[rr] * dh[c];
    }
    double jp[6];
    for (int t = 0; t < 3; ++t) {
        double ds[3];
        mat3_vec(dR + 9 * t, s, ds);
        jp[t] = sw * (nt[0] * ds[0] + nt[1] * ds[1] + nt[2] * ds[2]);
        jp[3 + t] = sw * nt[t];
    }
    double *gpose = Q->g + 12 * (size_t)m;
    for (int k = 0; k < K; ++k) {
        int j = idx[k];
        for (int l = 0; l < K; ++l)
            outer12(block_at(Q, j, idx[l]), a[k], a[l], 1.0);
        for (int p = 0; p < 12; ++p)
            Q->g[12 * (size_t)j + p] += r * a[k][p];
        for (int t = 0; t < 6; ++t)
            for (int p = 0; p < 12; ++p)
                Q->C[72 * (size_t)j + 12 * t + p] += jp[t] * a[k][p];
    }
    for (int t = 0; t < 6; ++t) {
        gpose[t] += r * jp[t];
        for (int u = 0; u < 6; ++u)
            Q->Hpp[6 * t + u] += jp[t] * jp[u];
    }
}

#ifdef _OPENMP
/* the data term of the OpenMP build: thread t sums the points of its
   contiguous range into its own normal equations (same pattern), then the
   thread sums are added to Q in thread order */
static void data_term_parallel(or_normal_eq *Q, const or_problem *P, const double *R, const double *dR,
                               const int *pix, const double *wpos, const double *spre)
{
    const int T = omp_get_max_threads(), N = P->N, K = P->K, m = Q->m;
    const size_t nblk = (size_t)Q->nnzb * 144, nC = (size_t)m * 72, ng = (size_t)12 * m + 6;
    or_normal_eq *S = (or_normal_eq *)calloc((size_t)T, sizeof(or_normal_eq));
    for (int t = 0; t < T; ++t) {
        S[t].m = m;
        S[t].nnzb = Q->nnzb;
        S[t].row_ptr = Q->row_ptr;
        S[t].col = Q->col;
        S[t].blk = (double *)calloc(nblk + 1, sizeof(double));
        S[t].C = (double *)calloc(nC + 1, sizeof(double));
        S[t].g = (double *)calloc(ng, sizeof(double));
    }
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int i0 = (int)((long)N * t / T), i1 = (int)((long)N * (t + 1) / T);
        or_normal_eq *St = S + t;
        for (int i = i0; i < i1; ++i) {
            if (pix[i] < 0) continue;
            double nt[3];
            double sw = sqrt(P->w_data);
            double r = sw * data_residual(P, pix[i], wpos + 3 * (size_t)i, nt);
            St->E[0] += r * r;
            St->n_valid++;
            add_plane_residual(St, P, R, dR, r, sw, nt, P->pos + 4 * (size_t)i, P->idx + (size_t)i * K,
                               P->w + (size_t)i * K, spre + 3 * (size_t)i);
        }
    }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < (long)nblk; ++e) {
        double v = Q->blk[e];
        for (int t = 0; t < T; ++t) v += S[t].blk[e];
        Q->blk[e] = v;
    }
    for (size_t e = 0; e < nC; ++e)
        for (int t = 0; t < T; ++t) Q->C[e] += S[t].C[e];
    for (size_t e = 0; e < ng; ++e)
        for (int t = 0; t < T; ++t) Q->g[e] += S[t].g[e];
    for (int t = 0; t < T; ++t) {
        for (int e = 0; e < 36; ++e) Q->Hpp[e] += S[t].Hpp[e];
        Q->E[0] += S[t].E[0];
        Q->n_valid += S[t].n_valid;
        free(S[t].blk);
        free(S[t].C);
        free(S[t].g);
    }
    free(S);
}
#endif

/*
 * Linearise Eq. (3) at (x, pose): association (or the frozen pix[] when
 * pix_in != NULL), residuals, energy terms, H = J^T J and g = J^T r with every
 * residual carrying sqrt(w) of its term.  pix_out (optional) receives the
 * association used.
 */
int or_linearize(const or_problem *P, const double *x, const double *pose, const int *pix_in, int *pix_out,
                 or_normal_eq *Q)
{
    int N = P->N, m = P->m, K = P->K;
    pattern_build(P, Q);
    double *wpos = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *wnrm = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *spre = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    int *pix = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    or_warp(P, x, pose, wpos, wnrm, spre);
    if (pix_in)
        memcpy(pix, pix_in, sizeof(int) * (size_t)N);
    else
        associate_from_f64(P, wpos, wnrm, pix);
    if (pix_out)
        memcpy(pix_out, pix, sizeof(int) * (size_t)N);
    double R[9], dR[27];
    or_rotation(pose, R, dR);
    double *gpose = Q->g + 12 * (size_t)m;

    /* data term */
#ifdef _OPENMP
    data_term_parallel(Q, P, R, dR, pix, wpos, spre);
#else
    for (int i = 0; i < N; ++i) {
        if (pix[i] < 0) continue;
        double nt[3];
        double sw = sqrt(P->w_data);
        double r = sw * data_residual(P, pix[i], wpos + 3 * (size_t)i, nt);
        Q->E[0] += r * r;
        Q->n_valid++;
        add_plane_residual(Q, P, R, dR, r, sw, nt, P->pos + 4 * (size_t)i, P->idx + (size_t)i * K,
                           P->w + (size_t)i * K, spre + 3 * (size_t)i);
    }
#endif

    /* E_corr: the three components of sqrt(w_corr) (v~_k - V_k) of every key
       point, each the residual of the plane through V_k normal to a camera axis */
    for (int k = 0; k < P->NK; ++k) {
        double vt[3], sk[3];
        warp_keypoint(P, x, R, pose, k, vt, sk);
        double sw = sqrt(P->w_corr);
        for (int c = 0; c < 3; ++c) {
            double nt[3] = {0.0, 0.0, 0.0};
            nt[c] = 1.0;
            double r = sw * (vt[c] - P->kp_tgt[3 * (size_t)k + c]);
            Q->E[5] += r * r;
            add_plane_residual(Q, P, R, dR, r, sw, nt, P->kp_pos + 4 * (size_t)k, P->kp_idx + (size_t)k * K,
                               P->kp_w + (size_t)k * K, sk);
        }
    }

    /* E_rot: Rot(A_j) on every node */
    for (int j = 0; j < m; ++j) {
        double rho[6], J[72];
        rot_residuals(x + 12 * (size_t)j, rho, J);
        double *bjj = block_at(Q, j, j);
        for (int q = 0; q < 6; ++q) {
            Q->E[1] += P->w_rot * rho[q] * rho[q];
            outer12(bjj, J + 12 * q, J + 12 * q, P->w_rot);
            for (int p = 0; p < 12; ++p)
                Q->g[12 * (size_t)j + p] += P->w_rot * rho[q] * J[12 * q + p];
        }
    }

    /* E_reg: alpha_jk = 1 on every directed edge j -> k of N(j) */
    for (int j = 0; j < m; ++j)
        for (int s = 0; s < P->KG; ++s) {
            int k = P->nbr[(size_t)j * P->KG + s];
            if (k < 0) continue;
            const double *gj = P->g + 4 * (size_t)j, *gk = P->g + 4 * (size_t)k;
            double e[3];
            reg_residual(x + 12 * (size_t)j, x + 12 * (size_t)k, gj, gk, e);
            double hh[4] = {gk[0] - gj[0], gk[1] - gj[1], gk[2] - gj[2], 1.0};
            for (int r = 0; r < 3; ++r) {
                double Jj[12] = {0}, Jk[12] = {0};
                for (int c = 0; c < 4; ++c) Jj[4 * r + c] = hh[c];
                Jk[4 * r + 3] = -1.0;
                Q->E[2] += P->w_reg * e[r] * e[r];
                outer12(block_at(Q, j, j), Jj, Jj, P->w_reg);
                outer12(block_at(Q, j, k), Jj, Jk, P->w_reg);
                outer12(block_at(Q, k, j), Jk, Jj, P->w_reg);
                outer12(block_at(Q, k, k), Jk, Jk, P->w_reg);
                for (int p = 0; p < 12; ++p) {
                    Q->g[12 * (size_t)j + p] += P->w_reg * e[r] * Jj[p];
                    Q->g[12 * (size_t)k + p] += P->w_reg * e[r] * Jk[p];
                }
            }
        }

    /* E_r, E_p: pose priors */
    for (int t = 0; t < 6; ++t) {
        double wt = t < 3 ? P->w_r : P->w_p;
        double d = pose[t] - P->prior[t];
        Q->E[t < 3 ? 3 : 4] += wt * d * d;
        Q->Hpp[6 * t + t] += wt;
        gpose[t] += wt * d;
    }
    free(wpos);
    free(wnrm);
    free(spre);
    free(pix);
    return OR_OK;
}

/* total energy (Eq. 3) at (x, pose) */
double or_energy(const or_problem *P, const double *x, const double *pose, const int *pix_in, double *terms,
                 int *n_valid)
{
    or_normal_eq Q;
    or_linearize(P, x, pose, pix_in, NULL, &Q);
    double E = Q.E[0] + Q.E[1] + Q.E[2] + Q.E[3] + Q.E[4] + Q.E[5];
    if (terms) memcpy(terms, Q.E, sizeof(Q.E));
    if (n_valid) *n_valid = Q.n_valid;
    or_normal_eq_free(&Q);
    return E;
}

/* ------------------------------------------------------------------------- */
/* Residual vector and explicit Jacobian (small problems, pins)               */
/* ------------------------------------------------------------------------- */

/* number of residual rows: valid data points, 6 per node, 3 per edge, 6 */
int or_residual_count(const or_problem *P, const int *pix)
{
    int n = 0;
    for (int i = 0; i < P->N; ++i) n += pix[i] >= 0;
    int ne = 0;
    for (int j = 0; j < P->m * P->KG; ++j) ne += P->nbr[j] >= 0;
    return n + 3 * P->NK + 6 * P->m + 3 * ne + 6;
}

/*
 * r (sqrt-weighted) and, when J != NULL, the dense Jacobian (rows x (12m+6))
 * with the association frozen to pix.  The Jacobian is written entry by entry
 * from the derivative of each residual formula.
 */
void or_residuals(const or_problem *P, const double *x, const double *pose, const int *pix, double *res,
                  double *J)
{
    int N = P->N, m = P->m, K = P->K;
    int ncol = 12 * m + 6;
    double *wpos = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *spre = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    or_warp(P, x, pose, wpos, NULL, spre);
    double R[9], dR[27];
    or_rotation(pose, R, dR);
    int row = 0;
    double sw = sqrt(P->w_data);
    for (int i = 0; i < N; ++i) {
        if (pix[i] < 0) continue;
        double nt[3];
        res[row] = sw * data_residual(P, pix[i], wpos + 3 * (size_t)i, nt);
        if (J) {
            double *Jr = J + (size_t)row * ncol;
            memset(Jr, 0, sizeof(double) * ncol);
            /* d v~ / d A_j[r][c] = w_j R e_r (v - g_j)_c ; d v~ / d t_j[r] = w_j R e_r */
            const double *v = P->pos + 4 * (size_t)i;
            for (int k = 0; k < K; ++k) {
                int j = P->idx[(size_t)i * K + k];
                double wj = P->w[(size_t)i * K + k];
                const double *gj = P->g + 4 * (size_t)j;
                double dh[4] = {v[0] - gj[0], v[1] - gj[1], v[2] - gj[2], 1.0};
                for (int r = 0; r < 3; ++r) {
                    double nRe = nt[0] * R[r] + nt[1] * R[3 + r] + nt[2] * R[6 + r]; /* n . (R e_r) */
                    for (int c = 0; c < 4; ++c)
                        Jr[12 * j + 4 * r + c] += sw * wj * nRe * dh[c];
                }
            }
            for (int t = 0; t < 3; ++t) {
                double ds[3];
                mat3_vec(dR + 9 * t, spre + 3 * (size_t)i, ds);
                Jr[12 * m + t] = sw * (nt[0] * ds[0] + nt[1] * ds[1] + nt[2] * ds[2]);
                Jr[12 * m + 3 + t] = sw * nt[t];
            }
        }
        row++;
    }
    /* E_corr rows: sqrt(w_corr) (v~_k - V_k), component c */
    double swc = sqrt(P->w_corr);
    for (int k = 0; k < P->NK; ++k) {
        double vt[3], sk[3];
        warp_keypoint(P, x, R, pose, k, vt, sk);
        const double *v = P->kp_pos + 4 * (size_t)k;
        for (int c = 0; c < 3; ++c) {
            res[row] = swc * (vt[c] - P->kp_tgt[3 * (size_t)k + c]);
            if (J) {
                double *Jr = J + (size_t)row * ncol;
                memset(Jr, 0, sizeof(double) * ncol);
                /* d v~_c / d A_j[r][c'] = w_j R[c][r] (v - g_j)_c' ; d v~_c / d t_j[r] = w_j R[c][r] */
                for (int q = 0; q < K; ++q) {
                    int j = P->kp_idx[(size_t)k * K + q];
                    double wj = P->kp_w[(size_t)k * K + q];
                    const double *gj = P->g + 4 * (size_t)j;
                    double dh[4] = {v[0] - gj[0], v[1] - gj[1], v[2] - gj[2], 1.0};
                    for (int r = 0; r < 3; ++r)
                        for (int cc = 0; cc < 4; ++cc)
                            Jr[12 * j + 4 * r + cc] += swc * wj * R[3 * c + r] * dh[cc];
                }
                for (int t = 0; t < 3; ++t) {
                    double ds[3];
                    mat3_vec(dR + 9 * t, sk, ds);
                    Jr[12 * m + t] = swc * ds[c];
                }
                Jr[12 * m + 3 + c] = swc;
            }
            row++;
        }
    }
    double swr = sqrt(P->w_rot);
    for (int j = 0; j < m; ++j) {
        double rho[6], Jq[72];
        rot_residuals(x + 12 * (size_t)j, rho, Jq);
        for (int q = 0; q < 6; ++q) {
            res[row] = swr * rho[q];
            if (J) {
                double *Jr = J + (size_t)row * ncol;
                memset(Jr, 0, sizeof(double) * ncol);
                for (int p = 0; p < 12; ++p) Jr[12 * j + p] = swr * Jq[12 * q + p];
            }
            row++;
        }
    }
    double swg = sqrt(P->w_reg);
    for (int j = 0; j < m; ++j)
        for (int s = 0; s < P->KG; ++s) {
            int k = P->nbr[(size_t)j * P->KG + s];
            if (k < 0) continue;
            const double *gj = P->g + 4 * (size_t)j, *gk = P->g + 4 * (size_t)k;
            double e[3];
            reg_residual(x + 12 * (size_t)j, x + 12 * (size_t)k, gj, gk, e);
            for (int r = 0; r < 3; ++r) {
                res[row] = swg * e[r];
                if (J) {
                    double *Jr = J + (size_t)row * ncol;
                    memset(Jr, 0, sizeof(double) * ncol);
                    for (int c = 0; c < 3; ++c) Jr[12 * j + 4 * r + c] = swg * (gk[c] - gj[c]);
                    Jr[12 * j + 4 * r + 3] += swg;
                    Jr[12 * k + 4 * r + 3] -= swg;
                }
                row++;
            }
        }
    for (int t = 0; t < 6; ++t) {
        double s = sqrt(t < 3 ? P->w_r : P->w_p);
        res[row] = s * (pose[t] - P->prior[t]);
        if (J) {
            double *Jr = J + (size_t)row * ncol;
            memset(Jr, 0, sizeof(double) * ncol);
            Jr[12 * m + t] = s;
        }
        row++;
    }
    free(wpos);
    free(spre);
}

/* ------------------------------------------------------------------------- */
/* Linear solvers                                                             */
/* ------------------------------------------------------------------------- */

/* in-place Cholesky A = L L^T of an n x n SPD matrix; returns 0 on success */
static int cholesky(double *A, int n)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / d;
        }
    }
    return 0;
}

static void chol_solve(const double *L, int n, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

/* dense P x P matrix of the normal equations (small problems) */
void or_normal_eq_dense(const or_normal_eq *Q, double *Hd)
{
    int m = Q->m, n = 12 * m + 6;
    memset(Hd, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < m; ++j)
        for (int t = Q->row_ptr[j]; t < Q->row_ptr[j + 1]; ++t) {
            int l = Q->col[t];
            for (int p = 0; p < 12; ++p)
                for (int q = 0; q < 12; ++q)
                    Hd[(size_t)(12 * j + p) * n + 12 * l + q] = Q->blk[144 * (size_t)t + 12 * p + q];
        }
    for (int j = 0; j < m; ++j)
        for (int t = 0; t < 6; ++t)
            for (int p = 0; p < 12; ++p) {
                double c = Q->C[72 * (size_t)j + 12 * t + p];
                Hd[(size_t)(12 * m + t) * n + 12 * j + p] = c;
                Hd[(size_t)(12 * j + p) * n + 12 * m + t] = c;
            }
    for (int t = 0; t < 6; ++t)
        for (int u = 0; u < 6; ++u)
            Hd[(size_t)(12 * m + t) * n + 12 * m + u] = Q->Hpp[6 * t + u];
}

/* LM damping: the diagonal of H scaled by (1 + lambda) */
static void damp(or_normal_eq *Q, double lambda)
{
    if (lambda == 0.0) return;
    for (int j = 0; j < Q->m; ++j) {
        double *b = block_at(Q, j, j);
        for (int p = 0; p < 12; ++p) b[13 * p] *= 1.0 + lambda;
    }
    for (int t = 0; t < 6; ++t) Q->Hpp[7 * t] *= 1.0 + lambda;
}

/* q = H p over the block pattern, the pose-node blocks and the pose block */
static void spmv(const or_normal_eq *Q, const double *p, double *q)
{
    int m = Q->m;
    const double *pp = p + 12 * (size_t)m;
    double *qp = q + 12 * (size_t)m;
    for (int t = 0; t < 6; ++t) qp[t] = 0.0;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < m; ++j) {
        double *qj = q + 12 * (size_t)j;
        for (int r = 0; r < 12; ++r) qj[r] = 0.0;
        for (int t = Q->row_ptr[j]; t < Q->row_ptr[j + 1]; ++t) {
            const double *b = Q->blk + 144 * (size_t)t;
            const double *pl = p + 12 * (size_t)Q->col[t];
            for (int r = 0; r < 12; ++r)
                for (int c = 0; c < 12; ++c) qj[r] += b[12 * r + c] * pl[c];
        }
        const double *C = Q->C + 72 * (size_t)j;
        for (int r = 0; r < 12; ++r)
            for (int t = 0; t < 6; ++t) qj[r] += C[12 * t + r] * pp[t];
    }
    for (int j = 0; j < m; ++j) {   /* the pose rows: sum over the nodes in order */
        const double *C = Q->C + 72 * (size_t)j;
        for (int t = 0; t < 6; ++t)
            for (int r = 0; r < 12; ++r) qp[t] += C[12 * t + r] * p[12 * (size_t)j + r];
    }
    for (int t = 0; t < 6; ++t)
        for (int u = 0; u < 6; ++u) qp[t] += Q->Hpp[6 * t + u] * pp[u];
}

static double dotv(const double *a, const double *b, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Block-Jacobi preconditioned CG on H d = b, x0 = 0, at most n_iter
 * iterations (early stop when tol > 0 and ||r|| <= tol ||b||).  The
 * preconditioner is the inverse of every 12x12 node block and of the 6x6
 * pose block, each shifted by jitter * trace / size before its Cholesky
 * factorisation.  Stops with OR_ERR_BREAKDOWN when p^T H p <= 0.
 * Returns the status; *iters = iterations done; res_hist (optional, n_iter+1)
 * receives ||r|| before each iteration and after the last.
 */
int or_pcg(const or_normal_eq *Q, const double *b, int n_iter, double tol, double jitter, double *d, int *iters,
           double *res_hist)
{
    int m = Q->m;
    size_t n = 12 * (size_t)m + 6;
    double *L = (double *)malloc(sizeof(double) * ((size_t)144 * m + 36));
    for (int j = 0; j < m; ++j) {
        double *Lj = L + 144 * (size_t)j;
        memcpy(Lj, block_at((or_normal_eq *)Q, j, j), sizeof(double) * 144);
        double tr = 0.0;
        for (int p = 0; p < 12; ++p) tr += Lj[13 * p];
        for (int p = 0; p < 12; ++p) Lj[13 * p] += jitter * tr / 12.0;
        if (cholesky(Lj, 12)) { free(L); return OR_ERR_BREAKDOWN; }
    }
    double *Lp = L + 144 * (size_t)m;
    {
        memcpy(Lp, Q->Hpp, sizeof(double) * 36);
        double tr = 0.0;
        for (int t = 0; t < 6; ++t) tr += Lp[7 * t];
        for (int t = 0; t < 6; ++t) Lp[7 * t] += jitter * tr / 6.0;
        if (cholesky(Lp, 6)) { free(L); return OR_ERR_BREAKDOWN; }
    }
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
#define PRECOND(dst, src)                                                                  \
    do {                                                                                   \
        for (int j_ = 0; j_ < m; ++j_)                                                     \
            chol_solve(L + 144 * (size_t)j_, 12, (src) + 12 * (size_t)j_, (dst) + 12 * (size_t)j_); \
        chol_solve(Lp, 6, (src) + 12 * (size_t)m, (dst) + 12 * (size_t)m);               \
    } while (0)
    for (size_t i = 0; i < n; ++i) { d[i] = 0.0; r[i] = b[i]; }
    PRECOND(z, r);
    for (size_t i = 0; i < n; ++i) p[i] = z[i];
    double rz = dotv(r, z, n);
    double bn = sqrt(dotv(b, b, n));
    int status = OR_OK, it = 0;
    if (res_hist) res_hist[0] = bn;
    for (it = 0; it < n_iter; ++it) {
        if (!(rz > 0.0)) break;           /* r == 0: exact solution reached */
        if (tol > 0.0 && sqrt(dotv(r, r, n)) <= tol * bn) break;
        spmv(Q, p, q);
        double pq = dotv(p, q, n);
        if (!(pq > 0.0)) { status = OR_ERR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (size_t i = 0; i < n; ++i) { d[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        PRECOND(z, r);
        double rz2 = dotv(r, z, n);
        double beta = rz2 / rz;
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz2;
        if (res_hist) res_hist[it + 1] = sqrt(dotv(r, r, n));
    }
#undef PRECOND
    if (iters) *iters = it;
    free(L); free(r); free(z); free(p); free(q);
    return status;
}

/* dense Cholesky solve of H d = b (tiny problems) */
int or_dense_solve(const or_normal_eq *Q, const double *b, double *d)
{
    int n = 12 * Q->m + 6;
    double *H = (double *)malloc(sizeof(double) * (size_t)n * n);
    or_normal_eq_dense(Q, H);
    int st = cholesky(H, n);
    if (!st) chol_solve(H, n, b, d);
    free(H);
    return st ? OR_ERR_BREAKDOWN : OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Newton / Levenberg-Marquardt driver (Sec. II.F)                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n_gn, n_pcg;
    double pcg_tol, jitter;
    double lambda;       /* initial damping (0 = plain Gauss-Newton) */
    int lm_accept;       /* 1: roll back a step that raised the energy, lambda *= 10 */
    int dense;           /* 1: dense Cholesky instead of PCG */
} or_solver;

/*
 * n_gn iterations; each: linearise at the current (x, pose) with
 * re-association, record the energy, solve (H + lambda diag H) d = -g, update.
 * energy_hist[it*6 + 0..4] = energy terms at the start of iteration it,
 * [it*6 + 5] = number of valid data points.
 */
int or_gn_solve(const or_problem *P, const or_solver *S, double *x, double *pose, double *energy_hist)
{
    int m = P->m;
    size_t n = 12 * (size_t)m + 6;
    double *b = (double *)malloc(sizeof(double) * n), *d = (double *)malloc(sizeof(double) * n);
    double *xprev = (double *)malloc(sizeof(double) * n);
    double Eprev = INFINITY, lambda = S->lambda;
    int status = OR_OK;
    for (int it = 0; it < S->n_gn; ++it) {
        or_normal_eq Q;
        or_linearize(P, x, pose, NULL, NULL, &Q);
        double E = Q.E[0] + Q.E[1] + Q.E[2] + Q.E[3] + Q.E[4] + Q.E[5];
        if (S->lm_accept && it > 0 && !(E <= Eprev)) {   /* a non-finite energy is not a decrease */
            /* reject the last step */
            or_normal_eq_free(&Q);
            memcpy(x, xprev, sizeof(double) * 12 * (size_t)m);
            memcpy(pose, xprev + 12 * (size_t)m, sizeof(double) * 6);
            lambda = lambda > 0 ? lambda * 10.0 : 1e-4;
            or_linearize(P, x, pose, NULL, NULL, &Q);
            E = Q.E[0] + Q.E[1] + Q.E[2] + Q.E[3] + Q.E[4] + Q.E[5];
        } else if (S->lm_accept && it > 0) {
            lambda *= 0.1;
        }
        if (energy_hist) {
            for (int t = 0; t < 5; ++t) energy_hist[6 * it + t] = Q.E[t];
            energy_hist[6 * it + 5] = Q.n_valid;
        }
        damp(&Q, lambda);
        for (size_t i = 0; i < n; ++i) b[i] = -Q.g[i];
        int st = S->dense ? or_dense_solve(&Q, b, d) : or_pcg(&Q, b, S->n_pcg, S->pcg_tol, S->jitter, d, NULL, NULL);
        or_normal_eq_free(&Q);
        if (st != OR_OK) { status = st; break; }
        memcpy(xprev, x, sizeof(double) * 12 * (size_t)m);
        memcpy(xprev + 12 * (size_t)m, pose, sizeof(double) * 6);
        Eprev = E;
        for (size_t i = 0; i < 12 * (size_t)m; ++i) x[i] += d[i];
        for (int t = 0; t < 6; ++t) pose[t] += d[12 * (size_t)m + t];
    }
    free(b); free(d); free(xprev);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Model update (Sec. II.G, Algorithms 1-3, Eqs. fusion1-4)                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    float tau_d;          /* |z~ - D| gate, mm (Alg. 1 condition 1) */
    float cos_delta;      /* normal gate: dot > cos(delta) (Alg. 1 condition 2) */
    double omega_max;     /* Eq. fusion4 upper bound */
    int tau_time;         /* delete if frame - t > tau_time ... */
    double tau_weight;    /* ... and omega < tau_weight */
    int frame;            /* current frame index */
} or_fuse_params;

/*
 * Inputs: the model (pos: xyz + omega, nrm: xyz + stability, col, t) of
 * n_in points, already warped to the current frame (wpos/wnrm, FP32 from the
 * warp), and the frame (depth, nmap, colour).  Outputs the new model: kept
 * points in their original order, then the lifted pixels in pixel order.
 * Returns the output count or -1 when it would exceed capacity.
 *  1. Reg: each warped point projects to P(v~); per pixel the point of
 *     smallest z~ (then smallest index) wins -- a z-buffer (Alg. 2 step 2).
 *  2. Alg. 1: a pixel is registered when D(u) > 0, |z~ - D(u)| < tau_d and
 *     n~ . n(u) > cos(delta) for its Reg point (FP32 rule).
 *  3. Registered points fuse by Eqs. fusion1-4 with observation weight 1:
 *     D' = (z~ w + D)/(w+1) moves the point along its own ray (v~ D'/z~),
 *     colour and normal average the same way (normal renormalised),
 *     w' = min(w+1, omega_max), t = frame.
 *  4. Every other valid pixel (D > 0, normal valid) is lifted as a new point
 *     Pi(u, D) with n(u), colour, w = 1, t = frame (Group 2).
 *  5. An unregistered old point is deleted when frame - t > tau_time and
 *     w < tau_weight (Alg. 2 step 4 / Alg. 3); stability = (w >= tau_weight).
 */
int or_fuse(const float *pos, const float *nrm, const float *col, const int *tstamp, int n_in,
            const float *wpos, const float *wnrm, const float *depth, const float *nmap, const float *color,
            float fx, float fy, float cx, float cy, int W, int H, const or_fuse_params *F, int capacity,
            float *pos_out, float *nrm_out, float *col_out, int *t_out, int *reg_out)
{
    size_t npx = (size_t)W * H;
    uint64_t *zb = (uint64_t *)malloc(sizeof(uint64_t) * npx);
    int *reg = (int *)malloc(sizeof(int) * npx);
    unsigned char *fused = (unsigned char *)calloc((size_t)(n_in > 0 ? n_in : 1), 1);
    for (size_t q = 0; q < npx; ++q) zb[q] = UINT64_MAX;
    for (int i = 0; i < n_in; ++i) {
        const float *p = wpos + 4 * (size_t)i;
        int u, v;
        if (!project_f32(p[0], p[1], p[2], fx, fy, cx, cy, W, H, &u, &v)) continue;
        uint32_t zbits;
        memcpy(&zbits, &p[2], 4);
        uint64_t key = ((uint64_t)zbits << 32) | (uint32_t)i;
        size_t q = (size_t)v * W + u;
        if (key < zb[q]) zb[q] = key;
    }
    /* Algorithm 1 on every pixel of Reg */
    for (size_t q = 0; q < npx; ++q) {
        reg[q] = -1;
        if (zb[q] == UINT64_MAX) continue;
        int i = (int)(zb[q] & 0xffffffffu);
        float D = depth[q];
        if (!(D > 0.0f)) continue;
        const float *tn = nmap + 4 * q;
        if (tn[3] == 0.0f) continue;
        float dz = wpos[4 * (size_t)i + 2] - D;
        if (!(fabsf(dz) < F->tau_d)) continue;
        float c = dot3_f32(wnrm + 4 * (size_t)i, tn);
        if (!(c > F->cos_delta)) continue;
        reg[q] = i;
        fused[i] = 1;
    }
    if (reg_out) memcpy(reg_out, reg, sizeof(int) * npx);
    /* per registered point: its pixel (a point wins at most one pixel) */
    int *pix_of = (int *)malloc(sizeof(int) * (size_t)(n_in > 0 ? n_in : 1));
    for (int i = 0; i < n_in; ++i) pix_of[i] = -1;
    for (size_t q = 0; q < npx; ++q)
        if (reg[q] >= 0) pix_of[reg[q]] = (int)q;
    int n = 0;
    for (int i = 0; i < n_in; ++i) {
        const float *p = wpos + 4 * (size_t)i, *nn = wnrm + 4 * (size_t)i;
        double w = pos[4 * (size_t)i + 3];
        int t = tstamp[i];
        double P3[3] = {p[0], p[1], p[2]}, N3[3] = {nn[0], nn[1], nn[2]};
        double C4[4] = {col[4 * (size_t)i], col[4 * (size_t)i + 1], col[4 * (size_t)i + 2], col[4 * (size_t)i + 3]};
        if (fused[i]) {
            size_t q = (size_t)pix_of[i];
            double D = depth[q];
            double z = P3[2];
            double Df = (z * w + D) / (w + 1.0);
            for (int r = 0; r < 3; ++r) P3[r] = P3[r] * (Df / z);
            const float *tn = nmap + 4 * q, *tc = color + 4 * q;
            double Nf[3];
            for (int r = 0; r < 3; ++r) Nf[r] = (N3[r] * w + tn[r]) / (w + 1.0);
            double len = sqrt(Nf[0] * Nf[0] + Nf[1] * Nf[1] + Nf[2] * Nf[2]);
            for (int r = 0; r < 3; ++r) N3[r] = len > 0 ? Nf[r] / len : 0.0;
            for (int r = 0; r < 4; ++r) C4[r] = (C4[r] * w + tc[r]) / (w + 1.0);
            w = w + 1.0 < F->omega_max ? w + 1.0 : F->omega_max;
            t = F->frame;
        } else if (F->frame - t > F->tau_time && w < F->tau_weight) {
            continue; /* deleted */
        }
        if (n >= capacity) { n = -1; break; }
        for (int r = 0; r < 3; ++r) { pos_out[4 * (size_t)n + r] = (float)P3[r]; nrm_out[4 * (size_t)n + r] = (float)N3[r]; }
        pos_out[4 * (size_t)n + 3] = (float)w;
        nrm_out[4 * (size_t)n + 3] = w >= F->tau_weight ? 1.0f : 0.0f;
        for (int r = 0; r < 4; ++r) col_out[4 * (size_t)n + r] = (float)C4[r];
        t_out[n] = t;
        n++;
    }
    if (n >= 0) {
        for (size_t q = 0; q < npx; ++q) {
            if (reg[q] >= 0) continue;
            float D = depth[q];
            if (!(D > 0.0f) || nmap[4 * q + 3] == 0.0f) continue;
            if (n >= capacity) { n = -1; break; }
            int u = (int)(q % W), v = (int)(q / W);
            double d = D;
            pos_out[4 * (size_t)n] = (float)((u - (double)cx) * d / fx);
            pos_out[4 * (size_t)n + 1] = (float)((v - (double)cy) * d / fy);
            pos_out[4 * (size_t)n + 2] = D;
            pos_out[4 * (size_t)n + 3] = 1.0f;
            for (int r = 0; r < 3; ++r) nrm_out[4 * (size_t)n + r] = nmap[4 * q + r];
            nrm_out[4 * (size_t)n + 3] = 1.0f >= F->tau_weight ? 1.0f : 0.0f;
            for (int r = 0; r < 4; ++r) col_out[4 * (size_t)n + r] = color[4 * q + r];
            t_out[n] = F->frame;
            n++;
        }
    }
    free(zb); free(reg); free(fused); free(pix_of);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Point-cloud downsampling (Sec. III.A "a fixed box ... average points fill  */
/* inside each 3D box"; Alg. 3, first line)                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t key;
    int idx;
} or_key_idx;

static int cmp_key_idx(const void *a, const void *b)
{
    const or_key_idx *x = (const or_key_idx *)a, *y = (const or_key_idx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/*
 * Boxes of edge `box` anchored at the minimum of the points' bounding box.
 * Box index per axis in FP32: floor((x - min) / box) (one subtraction, one
 * division); boxes per axis floor((max - min) / box) + 1; key = ix + nx (iy +
 * ny iz).  The points of one box become one point (reading: the paper
 * averages the points in a box and says nothing of the other fields; here
 * the average is weighted by the fusion weight omega as in Eqs. fusion1-4,
 * the normal is the normalised weighted sum, the merged weight the capped sum
 * min(sum omega, omega_max), the time stamp the latest, the stability flag
 * omega >= tau_weight).  Output in increasing key order; returns the count,
 * -1 past capacity, -2 when the box grid has 2^32 boxes or more.
 */
int or_downsample(const float *pos, const float *nrm, const float *col, const int *tstamp, int n, float box,
                  double omega_max, double tau_weight, int capacity, float *pos_out, float *nrm_out, float *col_out,
                  int *t_out, uint32_t *key_out)
{
    if (n <= 0) return 0;
    float mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = pos[d]; mx[d] = pos[d]; }
    for (int i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            float v = pos[4 * (size_t)i + d];
            if (v < mn[d]) mn[d] = v;
            if (v > mx[d]) mx[d] = v;
        }
    long dims[3];
    for (int d = 0; d < 3; ++d) {
        float ext = mx[d] - mn[d];
        float q = ext / box;
        dims[d] = (long)floorf(q) + 1;
    }
    if ((double)dims[0] * (double)dims[1] * (double)dims[2] >= 4294967296.0) return -2;
    or_key_idx *ki = (or_key_idx *)malloc(sizeof(or_key_idx) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        long c[3];
        for (int d = 0; d < 3; ++d) {
            float rel = pos[4 * (size_t)i + d] - mn[d];
            float q = rel / box;
            c[d] = (long)floorf(q);
            if (c[d] > dims[d] - 1) c[d] = dims[d] - 1;
        }
        ki[i].key = (uint32_t)(c[0] + dims[0] * (c[1] + dims[1] * c[2]));
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(or_key_idx), cmp_key_idx);
    int out = 0;
    for (int a = 0; a < n;) {
        int b = a;
        while (b < n && ki[b].key == ki[a].key) ++b;
        double sw = 0, sp[3] = {0, 0, 0}, sn[3] = {0, 0, 0}, sc[4] = {0, 0, 0, 0};
        int tmax = tstamp[ki[a].idx];
        for (int k = a; k < b; ++k) {
            int i = ki[k].idx;
            double w = pos[4 * (size_t)i + 3];
            sw += w;
            for (int d = 0; d < 3; ++d) {
                sp[d] += w * pos[4 * (size_t)i + d];
                sn[d] += w * nrm[4 * (size_t)i + d];
            }
            for (int d = 0; d < 4; ++d) sc[d] += w * col[4 * (size_t)i + d];
            if (tstamp[i] > tmax) tmax = tstamp[i];
        }
        if (!(sw > 0)) {   /* no weight in the box: a plain average */
            sw = 0;
            for (int d = 0; d < 3; ++d) sp[d] = sn[d] = 0;
            for (int d = 0; d < 4; ++d) sc[d] = 0;
            for (int k = a; k < b; ++k) {
                int i = ki[k].idx;
                sw += 1.0;
                for (int d = 0; d < 3; ++d) { sp[d] += pos[4 * (size_t)i + d]; sn[d] += nrm[4 * (size_t)i + d]; }
                for (int d = 0; d < 4; ++d) sc[d] += col[4 * (size_t)i + d];
            }
        }
        if (out >= capacity) { free(ki); return -1; }
        double wsum = 0;
        for (int k = a; k < b; ++k) wsum += pos[4 * (size_t)ki[k].idx + 3];
        double w_out = wsum < omega_max ? wsum : omega_max;
        double len = sqrt(sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2]);
        for (int d = 0; d < 3; ++d) {
            pos_out[4 * (size_t)out + d] = (float)(sp[d] / sw);
            nrm_out[4 * (size_t)out + d] = (float)(len > 0 ? sn[d] / len : 0.0);
        }
        pos_out[4 * (size_t)out + 3] = (float)w_out;
        nrm_out[4 * (size_t)out + 3] = w_out >= tau_weight ? 1.0f : 0.0f;
        for (int d = 0; d < 4; ++d) col_out[4 * (size_t)out + d] = (float)(sc[d] / sw);
        t_out[out] = tmax;
        if (key_out) key_out[out] = ki[a].key;
        ++out;
        a = b;
    }
    free(ki);
    return out;
}

/*
 * Back-projection error (Sec. III: the projected model image minus the
 * observed depth image).  The model points (warped into the frame) are
 * projected by the FP32 rule P; a pixel keeps the point of smallest z, then
 * of lowest index; over the pixels that keep a point and have D > 0:
 * out = (sum |z - D|, count, max |z - D|, sum (z - D)^2).
 */
void or_depth_error(const float *wpos, int n, const float *depth, float fx, float fy, float cx, float cy, int W,
                    int H, double *out)
{
    size_t npx = (size_t)W * H;
    uint64_t *zb = (uint64_t *)malloc(sizeof(uint64_t) * npx);
    for (size_t q = 0; q < npx; ++q) zb[q] = UINT64_MAX;
    for (int i = 0; i < n; ++i) {
        const float *p = wpos + 4 * (size_t)i;
        int u, v;
        if (!project_f32(p[0], p[1], p[2], fx, fy, cx, cy, W, H, &u, &v)) continue;
        uint32_t zbits;
        memcpy(&zbits, &p[2], 4);
        uint64_t key = ((uint64_t)zbits << 32) | (uint32_t)i;
        size_t q = (size_t)v * W + u;
        if (key < zb[q]) zb[q] = key;
    }
    double sa = 0, cnt = 0, mx = 0, s2 = 0;
    for (size_t q = 0; q < npx; ++q) {
        if (zb[q] == UINT64_MAX) continue;
        double D = depth[q];
        if (!(D > 0)) continue;
        double z = wpos[4 * (size_t)(zb[q] & 0xffffffffu) + 2];
        double e = fabs(z - D);
        sa += e;
        cnt += 1;
        if (e > mx) mx = e;
        s2 += (z - D) * (z - D);
    }
    out[0] = sa;
    out[1] = cnt;
    out[2] = mx;
    out[3] = s2;
    free(zb);
}

/* ------------------------------------------------------------------------- */
/* exported accessors for the normal equations (Python side)                  */
/* ------------------------------------------------------------------------- */

or_normal_eq *or_normal_eq_new(void) { return (or_normal_eq *)calloc(1, sizeof(or_normal_eq)); }
void or_normal_eq_delete(or_normal_eq *Q) { if (Q) { or_normal_eq_free(Q); free(Q); } }
int or_normal_eq_nnzb(const or_normal_eq *Q) { return Q->nnzb; }
void or_normal_eq_export(const or_normal_eq *Q, int *row_ptr, int *col, double *blk, double *C, double *Hpp,
                         double *g, double *E, int *n_valid)
{
    int m = Q->m;
    if (row_ptr) memcpy(row_ptr, Q->row_ptr, sizeof(int) * ((size_t)m + 1));
    if (col) memcpy(col, Q->col, sizeof(int) * (size_t)Q->nnzb);
    if (blk) memcpy(blk, Q->blk, sizeof(double) * 144 * (size_t)Q->nnzb);
    if (C) memcpy(C, Q->C, sizeof(double) * 72 * (size_t)m);
    if (Hpp) memcpy(Hpp, Q->Hpp, sizeof(double) * 36);
    if (g) memcpy(g, Q->g, sizeof(double) * (12 * (size_t)m + 6));
    if (E) memcpy(E, Q->E, sizeof(double) * 6);
    if (n_valid) *n_valid = Q->n_valid;
}
int or_pcg_eq(const or_normal_eq *Q, const double *b, int n_iter, double tol, double jitter, double *d, int *iters,
              double *res_hist)
{
    return or_pcg(Q, b, n_iter, tol, jitter, d, iters, res_hist);
}
void or_damp(or_normal_eq *Q, double lambda) { damp(Q, lambda); }
