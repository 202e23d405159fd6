/*
 * Seeded synthetic tractography inputs for LiFE problems.
 *
 * This file holds only the input recipe: Fibonacci point sets for the gradient
 * and atom directions, persistent random walks through a voxel grid (optionally
 * restricted to an ellipsoidal mask), the raw COO list of Phi entries those walks
 * produce (duplicates NOT merged), a ground-truth weight vector and Gaussian
 * noise.  It contains none of the method's arithmetic: no dictionary, no
 * duplicate merging, no M*w or M^T*r.  Both the FP64 oracle and the CUDA
 * library consume exactly the arrays produced here.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Every fascicle owns an
 * independent stream keyed by (seed, fascicle), so results do not depend on
 * the OpenMP thread count.  Gaussians use the Box-Muller transform.
 *
 * Compile with -ffp-contract=off so that x86-64 and aarch64 builds round alike
 * (libm may still differ in the last bit on different machines).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } rng_t;

static inline uint64_t rng_next(rng_t* r) { r->s += GOLDEN_GAMMA; return mix64(r->s); }
/* uniform in [0,1) with 53 random bits */
static inline double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform in (0,1] */
static inline double rng_unif_pos(rng_t* r) { return ((double)(rng_next(r) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

static inline void rng_gauss2(rng_t* r, double* z0, double* z1) {
    double u1 = rng_unif_pos(r), u2 = rng_unif(r);
    double rad = sqrt(-2.0 * log(u1)), th = 6.283185307179586476925 * u2;
    *z0 = rad * cos(th);
    *z1 = rad * sin(th);
}

static inline rng_t rng_stream(uint64_t seed, uint64_t stream, uint64_t tag) {
    rng_t r;
    r.s = mix64(seed ^ mix64(stream * 0xD1B54A32D192ED03ULL + tag + 1));
    return r;
}

/* Fibonacci sphere: z_i = 1 - (2i+1)/n, phi_i = i * pi * (3 - sqrt 5). */
void synth_fibonacci_sphere(int n, double* xyz) {
    const double ga = 3.14159265358979323846 * (3.0 - sqrt(5.0));
    for (int i = 0; i < n; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / n;
        double rr = sqrt(fmax(0.0, 1.0 - z * z));
        double ph = ga * i;
        xyz[3 * i + 0] = rr * cos(ph);
        xyz[3 * i + 1] = rr * sin(ph);
        xyz[3 * i + 2] = z;
    }
}

/* Fibonacci hemisphere (z > 0): z_i = 1 - (i + 1/2)/n, same phi rule. */
void synth_fibonacci_hemisphere(int n, double* xyz) {
    const double ga = 3.14159265358979323846 * (3.0 - sqrt(5.0));
    for (int i = 0; i < n; ++i) {
        double z = 1.0 - (i + 0.5) / n;
        double rr = sqrt(fmax(0.0, 1.0 - z * z));
        double ph = ga * i;
        xyz[3 * i + 0] = rr * cos(ph);
        xyz[3 * i + 1] = rr * sin(ph);
        xyz[3 * i + 2] = z;
    }
}

/* Ellipsoid inscribed in the grid: voxel (i,j,k) is inside when its centre
 * satisfies sum(((c - n/2) / (n/2))^2) <= 1. */
static int in_ellipsoid(int i, int j, int k, int nx, int ny, int nz) {
    double x = (i + 0.5 - 0.5 * nx) / (0.5 * nx);
    double y = (j + 0.5 - 0.5 * ny) / (0.5 * ny);
    double z = (k + 0.5 - 0.5 * nz) / (0.5 * nz);
    return x * x + y * y + z * z <= 1.0;
}

/* Fills vox_id[nx*ny*nz] (raster order, x fastest) with the compact rank of the
 * voxel inside the mask, or -1 outside.  use_mask = 0 keeps every voxel.
 * Returns the number of voxels. */
int64_t synth_voxel_ids(int nx, int ny, int nz, int use_mask, int32_t* vox_id) {
    int64_t nv = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t lin = i + (int64_t)nx * (j + (int64_t)ny * k);
                int inside = use_mask ? in_ellipsoid(i, j, k, nx, ny, nz) : 1;
                vox_id[lin] = inside ? (int32_t)(nv++) : -1;
            }
    return nv;
}

/* Per-fascicle walk lengths, uniform integers in [lmin, lmax]. */
void synth_walk_lengths(uint64_t seed, int64_t nf, int lmin, int lmax, int32_t* len) {
    for (int64_t f = 0; f < nf; ++f) {
        rng_t r = rng_stream(seed, (uint64_t)f, 0);
        len[f] = lmin + (int32_t)(rng_next(&r) % (uint64_t)(lmax - lmin + 1));
    }
}

typedef struct {
    int nx, ny, nz;
    const int32_t* vox_id;
} grid_t;

static inline int64_t grid_voxel(const grid_t* g, const double p[3]) {
    if (!(p[0] >= 0.0 && p[1] >= 0.0 && p[2] >= 0.0)) return -1;
    int i = (int)floor(p[0]), j = (int)floor(p[1]), k = (int)floor(p[2]);
    if (i >= g->nx || j >= g->ny || k >= g->nz) return -1;
    return g->vox_id[i + (int64_t)g->nx * (j + (int64_t)g->ny * k)];
}

static inline void normalize3(double t[3]) {
    double n = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    if (n > 0) { t[0] /= n; t[1] /= n; t[2] /= n; }
    else { t[0] = 0; t[1] = 0; t[2] = 1; }
}

/* Nearest dictionary orientation to the tangent, antipodally symmetric:
 * argmax_a |t . u_a|, ties to the lowest a. */
static inline int nearest_atom(const double t[3], int na, const double* ux, const double* uy,
                               const double* uz, double* scratch) {
    for (int a = 0; a < na; ++a) scratch[a] = fabs(t[0] * ux[a] + t[1] * uy[a] + t[2] * uz[a]);
    int best = 0;
    double bv = scratch[0];
    for (int a = 1; a < na; ++a)
        if (scratch[a] > bv) { bv = scratch[a]; best = a; }
    return best;
}

/*
 * Persistent random walks.  Fascicle f starts at a point drawn uniformly inside
 * the (masked) grid with a direction uniform on the sphere.  Each of its len[f]
 * steps: t <- normalize(t + persist * xi), xi ~ N(0, I3); step length ~ U(lo, hi)
 * voxels; if the end point leaves the domain, the offending box coordinates of t
 * are reflected (box exit) or t is reflected about the ellipsoid normal (mask
 * exit); failing that, t is reversed; failing that, the step stays in place.
 * The step emits one raw Phi entry: voxel = voxel of the step midpoint (of the
 * end point if the midpoint falls outside the mask), atom = nearest orientation
 * to t, value = step length.  Entries are written at off[f] .. off[f]+len[f]-1.
 */
void synth_walks(uint64_t seed, int64_t nf, const int32_t* len, const int64_t* off,
                 int nx, int ny, int nz, const int32_t* vox_id, int use_mask,
                 int na, const double* atom_xyz, double persist, double step_lo, double step_hi,
                 int32_t* out_atom, int32_t* out_voxel, int32_t* out_fasc, float* out_val) {
    grid_t g = {nx, ny, nz, vox_id};
    double* ux = (double*)malloc(sizeof(double) * 3 * na);
    double* uy = ux + na;
    double* uz = uy + na;
    for (int a = 0; a < na; ++a) {
        ux[a] = atom_xyz[3 * a];
        uy[a] = atom_xyz[3 * a + 1];
        uz[a] = atom_xyz[3 * a + 2];
    }
    const double cx = 0.5 * nx, cy = 0.5 * ny, cz = 0.5 * nz;
#pragma omp parallel
    {
        double* scratch = (double*)malloc(sizeof(double) * na);
#pragma omp for schedule(dynamic, 256)
        for (int64_t f = 0; f < nf; ++f) {
            rng_t r = rng_stream(seed, (uint64_t)f, 1);
            double p[3], t[3], q[3], m[3], z0, z1, z2, z3;
            /* start point: rejection sampling inside the domain */
            for (int tries = 0;; ++tries) {
                p[0] = rng_unif(&r) * nx;
                p[1] = rng_unif(&r) * ny;
                p[2] = rng_unif(&r) * nz;
                if (grid_voxel(&g, p) >= 0 || tries > 100000) break;
            }
            rng_gauss2(&r, &z0, &z1);
            rng_gauss2(&r, &z2, &z3);
            t[0] = z0; t[1] = z1; t[2] = z2;
            normalize3(t);
            int64_t o = off[f];
            for (int s = 0; s < len[f]; ++s) {
                rng_gauss2(&r, &z0, &z1);
                rng_gauss2(&r, &z2, &z3);
                t[0] += persist * z0;
                t[1] += persist * z1;
                t[2] += persist * z2;
                normalize3(t);
                double ell = step_lo + (step_hi - step_lo) * rng_unif(&r);
                for (int d = 0; d < 3; ++d) q[d] = p[d] + ell * t[d];
                if (grid_voxel(&g, q) < 0) {
                    /* box exit: reflect offending coordinates */
                    const int dims[3] = {nx, ny, nz};
                    int box_exit = 0;
                    for (int d = 0; d < 3; ++d)
                        if (q[d] < 0.0 || q[d] >= dims[d]) { t[d] = -t[d]; box_exit = 1; }
                    if (!box_exit && use_mask) {
                        /* mask exit: reflect about the ellipsoid normal at p */
                        double nrm[3] = {(p[0] - cx) / (cx * cx), (p[1] - cy) / (cy * cy), (p[2] - cz) / (cz * cz)};
                        normalize3(nrm);
                        double tn = t[0] * nrm[0] + t[1] * nrm[1] + t[2] * nrm[2];
                        for (int d = 0; d < 3; ++d) t[d] -= 2.0 * tn * nrm[d];
                    }
                    for (int d = 0; d < 3; ++d) q[d] = p[d] + ell * t[d];
                    if (grid_voxel(&g, q) < 0) {
                        for (int d = 0; d < 3; ++d) { t[d] = -t[d]; q[d] = p[d] + ell * t[d]; }
                        if (grid_voxel(&g, q) < 0)
                            for (int d = 0; d < 3; ++d) q[d] = p[d];
                    }
                }
                for (int d = 0; d < 3; ++d) m[d] = 0.5 * (p[d] + q[d]);
                int64_t v = grid_voxel(&g, m);
                if (v < 0) v = grid_voxel(&g, q);
                if (v < 0) v = grid_voxel(&g, p);
                out_atom[o + s] = nearest_atom(t, na, ux, uy, uz, scratch);
                out_voxel[o + s] = (int32_t)v;
                out_fasc[o + s] = (int32_t)f;
                out_val[o + s] = (float)ell;
                for (int d = 0; d < 3; ++d) p[d] = q[d];
            }
        }
        free(scratch);
    }
    free(ux);
}

/* Ground-truth weights: U(0,1), each fascicle zeroed with probability zero_frac. */
void synth_w_true(uint64_t seed, int64_t nf, double zero_frac, float* w) {
    for (int64_t f = 0; f < nf; ++f) {
        rng_t r = rng_stream(seed, (uint64_t)f, 2);
        double u = rng_unif(&r), z = rng_unif(&r);
        w[f] = z < zero_frac ? 0.0f : (float)u;
    }
}

/* Counter-based Gaussian noise, sigma * N(0,1) per entry; entry i uses stream
 * (seed, i/2, tag 3) so any slice can be regenerated independently. */
void synth_noise(uint64_t seed, int64_t n, double sigma, float* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i += 2) {
        rng_t r = rng_stream(seed, (uint64_t)(i / 2), 3);
        double z0, z1;
        rng_gauss2(&r, &z0, &z1);
        out[i] = (float)(sigma * z0);
        if (i + 1 < n) out[i + 1] = (float)(sigma * z1);
    }
}

/* Log-uniform integer in [lo, hi] and uniform integer in [lo, hi], for batched
 * problem shapes (stream tag 4 + k). */
int64_t synth_loguniform_int(uint64_t seed, int64_t k, int64_t lo, int64_t hi) {
    rng_t r = rng_stream(seed, (uint64_t)k, 4);
    double u = rng_unif(&r);
    double x = exp(log((double)lo) + u * (log((double)hi) - log((double)lo)));
    int64_t v = (int64_t)floor(x + 0.5);
    return v < lo ? lo : (v > hi ? hi : v);
}

int64_t synth_uniform_int(uint64_t seed, int64_t k, int64_t lo, int64_t hi) {
    rng_t r = rng_stream(seed, (uint64_t)k, 5);
    return lo + (int64_t)(rng_next(&r) % (uint64_t)(hi - lo + 1));
}
