/*
 * Voronoi cells by half-space clipping -- a seeded synthetic-mesh input
 * generator. It stands in for the moving-mesh code's own tessellation (the
 * method is defined on a Voronoi grid, paper Sec. 2.1 and Appendix A) and
 * holds none of the transport method's arithmetic: it only turns generator
 * points into cell volumes, face areas and neighbour pairs.
 *
 * Each cell starts as a box around its generator and is clipped by the
 * bisector plane of every candidate neighbour, nearest first. Clipping stops
 * once the next candidate is farther than twice the cell's radius (no farther
 * plane can cut the cell). Geometry is kept relative to the generator.
 *
 * Faces are convex polygons stored as vertex lists. A vertex created on an
 * edge is computed from the edge's (inside, outside) endpoints in that order,
 * so the two faces that share the edge create bit-identical copies of it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VOR_MAXF 128
#define VOR_MAXV 96

typedef struct {
    int nv;
    int32_t nbr;   /* neighbour generator (index into the original set), -1 = box wall */
    int32_t code;  /* periodic image code (0..26, 13 = none) or box wall id (0..5) */
    double hd;     /* distance from the generator to the face plane */
    double v[VOR_MAXV][3];
} vface;

typedef struct {
    int nf;
    vface f[VOR_MAXF];
    vface tmp;
} vcell;

enum { VOR_OK = 0, VOR_NEED_MORE = 1, VOR_OVERFLOW = 2, VOR_TOO_BIG = 3, VOR_COMPLEX = 4 };

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void init_box(vcell* c, const double lo[3], const double hi[3], int periodic) {
    /* six faces of the box [lo,hi] (relative coordinates); wall w = 2*axis + (0 low, 1 high) */
    c->nf = 0;
    for (int ax = 0; ax < 3; ++ax) {
        for (int side = 0; side < 2; ++side) {
            vface* f = &c->f[c->nf++];
            int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
            double x = side ? hi[ax] : lo[ax];
            double q[4][2] = {{lo[a1], lo[a2]}, {hi[a1], lo[a2]}, {hi[a1], hi[a2]}, {lo[a1], hi[a2]}};
            f->nv = 4;
            for (int k = 0; k < 4; ++k) {
                f->v[k][ax] = x;
                f->v[k][a1] = q[k][0];
                f->v[k][a2] = q[k][1];
            }
            f->hd = fabs(x);
            if (periodic) {
                int s[3] = {0, 0, 0};
                s[ax] = side ? 1 : -1;
                f->nbr = -2; /* the generator's own image; the caller relabels it */
                f->code = (s[0] + 1) + 3 * (s[1] + 1) + 9 * (s[2] + 1);
            } else {
                f->nbr = -1;
                f->code = 2 * ax + side;
            }
        }
    }
}

static double max_r2(const vcell* c) {
    double r2 = 0.0;
    for (int i = 0; i < c->nf; ++i)
        for (int k = 0; k < c->f[i].nv; ++k) {
            double q = dot3(c->f[i].v[k], c->f[i].v[k]);
            if (q > r2) r2 = q;
        }
    return r2;
}

/* clip by {p : p.d <= |d|^2/2}; returns 0 ok, -1 on capacity overflow */
static int clip(vcell* c, const double d[3], int32_t nbr, int32_t code) {
    const double h = 0.5 * dot3(d, d);
    int any_out = 0;
    for (int i = 0; i < c->nf && !any_out; ++i)
        for (int k = 0; k < c->f[i].nv; ++k)
            if (dot3(c->f[i].v[k], d) - h > 0.0) { any_out = 1; break; }
    if (!any_out) return 0;

    double cut[2 * VOR_MAXV][3];
    int ncut = 0;
    int nf_out = 0;
    for (int i = 0; i < c->nf; ++i) {
        vface* f = &c->f[i];
        double dist[VOR_MAXV];
        int nin = 0;
        for (int k = 0; k < f->nv; ++k) {
            dist[k] = dot3(f->v[k], d) - h;
            if (dist[k] <= 0.0) ++nin;
        }
        if (nin == 0) continue; /* face removed */
        vface* g = &c->tmp;
        g->nv = 0;
        g->nbr = f->nbr;
        g->code = f->code;
        g->hd = f->hd;
        for (int k = 0; k < f->nv; ++k) {
            int k2 = (k + 1) % f->nv;
            int in1 = dist[k] <= 0.0, in2 = dist[k2] <= 0.0;
            if (in1) {
                if (g->nv >= VOR_MAXV) return -1;
                memcpy(g->v[g->nv++], f->v[k], sizeof(double) * 3);
                if (dist[k] == 0.0) {
                    if (ncut >= 2 * VOR_MAXV) return -1;
                    memcpy(cut[ncut++], f->v[k], sizeof(double) * 3);
                }
            }
            if (in1 != in2 && dist[k] != 0.0 && dist[k2] != 0.0) {
                const double* pin = in1 ? f->v[k] : f->v[k2];
                const double* pout = in1 ? f->v[k2] : f->v[k];
                double din = in1 ? dist[k] : dist[k2];
                double dout = in1 ? dist[k2] : dist[k];
                double t = din / (din - dout);
                double x[3];
                for (int a = 0; a < 3; ++a) x[a] = pin[a] + t * (pout[a] - pin[a]);
                if (g->nv >= VOR_MAXV || ncut >= 2 * VOR_MAXV) return -1;
                memcpy(g->v[g->nv++], x, sizeof x);
                memcpy(cut[ncut++], x, sizeof x);
            }
        }
        if (g->nv >= 3) {
            c->f[nf_out] = *g;
            ++nf_out;
        }
    }
    c->nf = nf_out;

    /* the new face: distinct cut points, ordered by angle around their centroid */
    double pts[2 * VOR_MAXV][3];
    int np = 0;
    for (int k = 0; k < ncut; ++k) {
        int dup = 0;
        for (int m = 0; m < np; ++m)
            if (pts[m][0] == cut[k][0] && pts[m][1] == cut[k][1] && pts[m][2] == cut[k][2]) { dup = 1; break; }
        if (!dup) memcpy(pts[np++], cut[k], sizeof(double) * 3);
    }
    if (np < 3) return 0;
    if (np > VOR_MAXV || c->nf >= VOR_MAXF) return -1;
    double ctr[3] = {0, 0, 0};
    for (int k = 0; k < np; ++k)
        for (int a = 0; a < 3; ++a) ctr[a] += pts[k][a] / np;
    double nrm = sqrt(dot3(d, d));
    double n[3] = {d[0] / nrm, d[1] / nrm, d[2] / nrm};
    double u[3];
    if (fabs(n[0]) < 0.6) { u[0] = 0; u[1] = n[2]; u[2] = -n[1]; }
    else { u[0] = -n[2]; u[1] = 0; u[2] = n[0]; }
    double un = sqrt(dot3(u, u));
    for (int a = 0; a < 3; ++a) u[a] /= un;
    double w[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
    double ang[2 * VOR_MAXV];
    for (int k = 0; k < np; ++k) {
        double r[3] = {pts[k][0] - ctr[0], pts[k][1] - ctr[1], pts[k][2] - ctr[2]};
        ang[k] = atan2(dot3(r, w), dot3(r, u));
    }
    for (int k = 1; k < np; ++k) { /* insertion sort by angle */
        double a = ang[k], p[3] = {pts[k][0], pts[k][1], pts[k][2]};
        int m = k - 1;
        while (m >= 0 && ang[m] > a) {
            ang[m + 1] = ang[m];
            memcpy(pts[m + 1], pts[m], sizeof(double) * 3);
            --m;
        }
        ang[m + 1] = a;
        memcpy(pts[m + 1], p, sizeof(double) * 3);
    }
    vface* f = &c->f[c->nf++];
    f->nv = np;
    f->nbr = nbr;
    f->code = code;
    f->hd = 0.5 * nrm;
    for (int k = 0; k < np; ++k) memcpy(f->v[k], pts[k], sizeof(double) * 3);
    return 0;
}

static double face_area(const vface* f) {
    double s[3] = {0, 0, 0};
    for (int k = 0; k < f->nv; ++k) {
        const double* a = f->v[k];
        const double* b = f->v[(k + 1) % f->nv];
        s[0] += a[1] * b[2] - a[2] * b[1];
        s[1] += a[2] * b[0] - a[0] * b[2];
        s[2] += a[0] * b[1] - a[1] * b[0];
    }
    return 0.5 * sqrt(dot3(s, s));
}

/*
 * Build cells [c_begin, c_end) of the generators pts[n][3] in the unit box.
 *   periodic = 0: vacuum box [0,1]^3, walls become faces with nbr = -1;
 *                 ext_pts = all generators (ext_orig = identity, ext_code = 13).
 *   periodic = 1: periodic unit box (faces towards the generator's own images get
 *                 nbr = -2); ext_pts[n_ext][3] holds the generators and
 *                 their ghost images (ext_orig = original index, ext_code = image
 *                 code); candidates index ext_pts. margin = ghost layer width.
 * cand[n][k]: candidate indices into ext_pts, nearest first.
 * Writes volume[c], nfaces[c], status[c] and face records (cell, nbr, code, area)
 * at out[*n_out ...], capacity cap. Returns 0, or 1 if the output capacity was exceeded.
 */
int vor_build(const double* pts, int64_t n, int periodic, const double* ext_pts, const int32_t* ext_orig,
              const int8_t* ext_code, double margin, const int32_t* cand, int32_t k, int64_t c_begin,
              int64_t c_end, double* volume, int32_t* nfaces, int32_t* status, int64_t cap, int32_t* out_cell,
              int32_t* out_nbr, int8_t* out_code, double* out_area, int64_t* n_out) {
    (void)n;
    vcell* c = (vcell*)malloc(sizeof(vcell));
    if (!c) return 2;
    int64_t w = 0;
    int rc = 0;
    for (int64_t i = c_begin; i < c_end; ++i) {
        const double* x = pts + 3 * i;
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (periodic) { lo[a] = -0.5; hi[a] = 0.5; }
            else { lo[a] = -x[a]; hi[a] = 1.0 - x[a]; }
        }
        init_box(c, lo, hi, periodic);
        int st = VOR_NEED_MORE;
        double r2 = max_r2(c);
        for (int j = 0; j < k; ++j) {
            int32_t q = cand[i * (int64_t)k + j];
            if (q < 0) break;
            const double* y = ext_pts + 3 * (int64_t)q;
            double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
            double dd = dot3(d, d);
            if (dd == 0.0) continue; /* the generator itself */
            if (dd > 4.0 * r2) { st = VOR_OK; break; }
            int32_t nb = ext_orig[q];
            int32_t code = ext_code[q];
            if (clip(c, d, nb, code) != 0) { st = VOR_COMPLEX; break; }
            r2 = max_r2(c);
        }
        if (st == VOR_OK && periodic && 2.0 * sqrt(r2) > margin) st = VOR_TOO_BIG;
        status[i] = st;
        double vol = 0.0;
        int nf = 0;
        for (int f = 0; f < c->nf; ++f) {
            double A = face_area(&c->f[f]);
            vol += A * c->f[f].hd / 3.0;
            if (A <= 0.0) continue;
            if (w >= cap) { rc = 1; break; }
            out_cell[w] = (int32_t)i;
            out_nbr[w] = c->f[f].nbr;
            out_code[w] = (int8_t)c->f[f].code;
            out_area[w] = A;
            ++w;
            ++nf;
        }
        volume[i] = vol;
        nfaces[i] = nf;
        if (rc) break;
    }
    *n_out = w;
    free(c);
    return rc;
}
