/*
 * FP64 CPU oracle for the LiFE hot path (test infrastructure only).
 *
 * Plain, slow, obviously correct loops written from the paper's definitions.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library; the product path (the CUDA library) shares no code with it.
 *
 *   oracle_dictionary  D[θ,a] = exp(-b λ (g_θ·u_a)^2), each column demeaned, and dD/dλ
 *                      (dictionary of canonical diffusion atoms, Eq. 3; the
 *                      exponential atom model and demeaning are the workload recipe)
 *   oracle_canon       restructured (sorted) Phi with duplicate (a,v,f) entries merged
 *                      (Sec. 4.1.2 data restructuring: atom-, voxel-, fiber-based)
 *   oracle_dsc         y = M w,   y[θ,v] = Σ_k D[θ,a_k] val_k w[f_k] [v_k = v]  (Eq. 1, Eq. 3-4)
 *   oracle_wc          g = M^T r, g[f] = Σ_k val_k Σ_θ D[θ,a_k] r[θ,v_k] [f_k = f]
 *   oracle_sbb_step    one SBB-NNLS iteration (Eq. 5-8, Algorithm 1)
 *   oracle_grad_D      dL/dD for L = ½‖r - M(D) w‖²
 *   oracle_voxel_rmse  per-voxel prediction error sqrt(Σ_θ e[θ,v]² / Nθ) of a residual
 *                      (the error by which LiFE evaluates a connectome, Sec. 2.1)
 *   oracle_prune       the pruned connectome: fascicles with weight above a threshold
 *                      (LiFE keeps the fascicles of positive weight, Sec. 1 and Sec. 2.1)
 *
 * Layouts: D is column-major D[θ + Nθ·a]; signals y, r, b, e are column-major
 * [θ + Nθ·v].  All arithmetic is double precision; compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- dictionary */

/* D_raw[θ,a] = exp(-bval·lam·(g_θ·u_a)^2); D = D_raw minus its column mean over θ.
 * dD[θ,a] = d D / d lam = (-bval c^2 exp(-bval lam c^2)) minus its column mean. */
void oracle_dictionary(int nt, int na, const double* g, const double* u, double bval, double lam,
                       double* D, double* dD) {
    for (int a = 0; a < na; ++a) {
        double mean = 0.0, dmean = 0.0;
        for (int t = 0; t < nt; ++t) {
            double c = g[3 * t] * u[3 * a] + g[3 * t + 1] * u[3 * a + 1] + g[3 * t + 2] * u[3 * a + 2];
            double e = exp(-bval * lam * c * c);
            D[t + (int64_t)nt * a] = e;
            mean += e;
            if (dD) {
                dD[t + (int64_t)nt * a] = -bval * c * c * e;
                dmean += dD[t + (int64_t)nt * a];
            }
        }
        mean /= nt;
        dmean /= nt;
        for (int t = 0; t < nt; ++t) {
            D[t + (int64_t)nt * a] -= mean;
            if (dD) dD[t + (int64_t)nt * a] -= dmean;
        }
    }
}

/* ---------------------------------------------------------- restructuring */

typedef struct { int32_t k1, k2, k3; int32_t idx; } key3_t;

static int cmp_key3(const void* pa, const void* pb) {
    const key3_t* a = (const key3_t*)pa;
    const key3_t* b = (const key3_t*)pb;
    if (a->k1 != b->k1) return a->k1 < b->k1 ? -1 : 1;
    if (a->k2 != b->k2) return a->k2 < b->k2 ? -1 : 1;
    if (a->k3 != b->k3) return a->k3 < b->k3 ? -1 : 1;
    return 0;
}

/*
 * Sort Phi by the chosen dimension and merge entries with equal (a,v,f).
 *   order 0: voxel-based   (v, a, f)
 *   order 1: fiber-based   (f, v, a)
 *   order 2: atom-based    (a, v, f)
 * Merged values are summed in double precision and rounded once to float.
 * Returns the number of distinct entries, or -1 if an index is out of range
 * or a value is not finite.
 */
int64_t oracle_canon(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                     const float* val, int32_t na, int32_t nv, int32_t nf, int order,
                     int32_t* oa, int32_t* ov, int32_t* of, float* oval) {
    for (int64_t i = 0; i < n; ++i) {
        if (atom[i] < 0 || atom[i] >= na || voxel[i] < 0 || voxel[i] >= nv || fasc[i] < 0 || fasc[i] >= nf)
            return -1;
        if (!isfinite(val[i])) return -1;
    }
    if (n == 0) return 0;
    key3_t* k = (key3_t*)malloc(sizeof(key3_t) * (size_t)n);
    if (!k) return -2;
    for (int64_t i = 0; i < n; ++i) {
        int32_t a = atom[i], v = voxel[i], f = fasc[i];
        if (order == 0) { k[i].k1 = v; k[i].k2 = a; k[i].k3 = f; }
        else if (order == 1) { k[i].k1 = f; k[i].k2 = v; k[i].k3 = a; }
        else { k[i].k1 = a; k[i].k2 = v; k[i].k3 = f; }
        k[i].idx = (int32_t)i;
    }
    qsort(k, (size_t)n, sizeof(key3_t), cmp_key3);
    int64_t m = 0;
    int64_t i = 0;
    while (i < n) {
        int64_t j = i;
        double s = 0.0;
        while (j < n && k[j].k1 == k[i].k1 && k[j].k2 == k[i].k2 && k[j].k3 == k[i].k3) {
            s += (double)val[k[j].idx];
            ++j;
        }
        int32_t a, v, f;
        if (order == 0) { v = k[i].k1; a = k[i].k2; f = k[i].k3; }
        else if (order == 1) { f = k[i].k1; v = k[i].k2; a = k[i].k3; }
        else { a = k[i].k1; v = k[i].k2; f = k[i].k3; }
        oa[m] = a; ov[m] = v; of[m] = f; oval[m] = (float)s;
        ++m;
        i = j;
    }
    free(k);
    return m;
}

/* ---------------------------------------------------------------- SpMVs */

/* DSC: y = M w.  For every nonzero, y[:,v] += D[:,a] * (val * w[f]) (the daxpy
 * of the paper's inner loop), y zeroed first. */
void oracle_dsc(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                const double* val, int nt, const double* D, const double* w, int64_t nv, double* y) {
    memset(y, 0, sizeof(double) * (size_t)nt * (size_t)nv);
    for (int64_t k = 0; k < n; ++k) {
        double s = val[k] * w[fasc[k]];
        const double* d = D + (int64_t)nt * atom[k];
        double* yv = y + (int64_t)nt * voxel[k];
        for (int t = 0; t < nt; ++t) yv[t] += d[t] * s;
    }
}

/* WC: g = M^T r.  For every nonzero, g[f] += val * <D[:,a], r[:,v]> (the dot of
 * the paper's inner loop), g zeroed first. */
void oracle_wc(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
               const double* val, int nt, const double* D, const double* r, int64_t nf, double* g) {
    memset(g, 0, sizeof(double) * (size_t)nf);
    for (int64_t k = 0; k < n; ++k) {
        const double* d = D + (int64_t)nt * atom[k];
        const double* rv = r + (int64_t)nt * voxel[k];
        double dot = 0.0;
        for (int t = 0; t < nt; ++t) dot += d[t] * rv[t];
        g[fasc[k]] += val[k] * dot;
    }
}

/* dL/dD for L = ½‖r - M(D) w‖² given the residual e = M w - r:
 * gD[θ,a] = Σ_k val_k w[f_k] e[θ, v_k] over nonzeros with a_k = a. */
void oracle_grad_D(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                   const double* val, int nt, int na, const double* w, const double* e, double* gD) {
    memset(gD, 0, sizeof(double) * (size_t)nt * (size_t)na);
    for (int64_t k = 0; k < n; ++k) {
        double s = val[k] * w[fasc[k]];
        const double* ev = e + (int64_t)nt * voxel[k];
        double* gd = gD + (int64_t)nt * atom[k];
        for (int t = 0; t < nt; ++t) gd[t] += ev[t] * s;
    }
}

/* ------------------------------------------------------------- SBB-NNLS */

typedef struct {
    int64_t it;        /* iterations taken so far (0-based index of the next one) */
    double alpha;      /* last step size (1 before the first step) */
    double obj;        /* ½‖M w - b‖² at the start of the last iteration */
    double gg;         /* <g~, g~> at the start of the last iteration */
    double gg0;        /* <g~, g~> at iteration 0 */
    double vv;         /* <M g~, M g~> */
    double uu;         /* <M^T M g~, M^T M g~> (Eq. 8 iterations only) */
    int32_t eq;        /* step rule used last: 7 or 8 (0 if none) */
    int32_t converged; /* 1 once ‖g~‖ <= tol ‖g~_0‖ or g~ = 0 */
} oracle_sbb_state;

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * One SBB-NNLS iteration (Eq. 5-8, Algorithm 1), in double precision:
 *   e  = M w - b,  obj = ½ <e,e>
 *   g  = M^T e                                  (Eq. 6)
 *   g~ = g with g~_f = 0 where w_f = 0 and g_f > 0   (projected / subspace gradient)
 *   stop if <g~,g~> = 0 or ‖g~‖ <= tol ‖g~_0‖
 *   v' = M g~
 *   iteration rule A (Eq. 7): alpha = <g~,g~> / <v',v'>
 *   iteration rule B (Eq. 8): alpha = <v',v'> / <v'',v''>, v'' = M^T v'
 *   rule A on even 0-based iterations when eq7_on_even, else on odd ones;
 *   a zero denominator keeps the previous alpha.
 *   w <- [w - alpha g~]_+                        (Eq. 5)
 * work must hold 2*nt*nv + 2*nf doubles.
 */
void oracle_sbb_step(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                     const double* val, int nt, const double* D, int64_t nv, int64_t nf,
                     const double* b, double* w, double tol, int eq7_on_even,
                     oracle_sbb_state* st, double* work) {
    if (st->converged) return;
    int64_t ny = (int64_t)nt * nv;
    double* e = work;
    double* v = work + ny;
    double* g = work + 2 * ny;
    double* u = g + nf;
    oracle_dsc(n, atom, voxel, fasc, val, nt, D, w, nv, e);
    for (int64_t i = 0; i < ny; ++i) e[i] -= b[i];
    st->obj = 0.5 * dot(ny, e, e);
    oracle_wc(n, atom, voxel, fasc, val, nt, D, e, nf, g);
    for (int64_t f = 0; f < nf; ++f)
        if (w[f] == 0.0 && g[f] > 0.0) g[f] = 0.0;
    double gg = dot(nf, g, g);
    st->gg = gg;
    if (st->it == 0) st->gg0 = gg;
    if (gg == 0.0 || sqrt(gg) <= tol * sqrt(st->gg0)) {
        st->converged = 1;
        st->eq = 0;
        return;
    }
    oracle_dsc(n, atom, voxel, fasc, val, nt, D, g, nv, v);
    double vv = dot(ny, v, v);
    st->vv = vv;
    int even = (st->it % 2) == 0;
    int use7 = eq7_on_even ? even : !even;
    double alpha = st->alpha;
    if (use7) {
        st->eq = 7;
        st->uu = 0.0;
        if (vv > 0.0) alpha = gg / vv;
    } else {
        st->eq = 8;
        oracle_wc(n, atom, voxel, fasc, val, nt, D, v, nf, u);
        double uu = dot(nf, u, u);
        st->uu = uu;
        if (uu > 0.0) alpha = vv / uu;
    }
    st->alpha = alpha;
    for (int64_t f = 0; f < nf; ++f) {
        double x = w[f] - alpha * g[f];
        w[f] = x > 0.0 ? x : 0.0;
    }
    st->it += 1;
}

/* Runs up to max_iter iterations from the given w (state must be zeroed with
 * alpha = 1 by the caller on the first call). */
void oracle_sbb_solve(int64_t n, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                      const double* val, int nt, const double* D, int64_t nv, int64_t nf,
                      const double* b, double* w, double tol, int eq7_on_even, int64_t max_iter,
                      oracle_sbb_state* st, double* work) {
    for (int64_t i = 0; i < max_iter && !st->converged; ++i)
        oracle_sbb_step(n, atom, voxel, fasc, val, nt, D, nv, nf, b, w, tol, eq7_on_even, st, work);
}

/* ------------------------------------------------------------ evaluation */

/* Per-voxel root-mean-square of a residual e = M w - b over the Nθ directions:
 * rmse[v] = sqrt( Σ_θ e[θ,v]^2 / Nθ ).  Returns Σ over all (θ,v) of e^2. */
double oracle_voxel_rmse(int nt, int64_t nv, const double* e, double* rmse) {
    double total = 0.0;
    for (int64_t v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += e[t + (int64_t)nt * v] * e[t + (int64_t)nt * v];
        rmse[v] = sqrt(s / nt);
        total += s;
    }
    return total;
}

/* Pruned connectome: keep[f] = 1 when w[f] > threshold (a NaN weight is not
 * kept), kept[] = the kept fascicles in increasing order.  Returns their number. */
int64_t oracle_prune(int64_t nf, const float* w, float threshold, uint8_t* keep, int32_t* kept) {
    int64_t n = 0;
    for (int64_t f = 0; f < nf; ++f) {
        keep[f] = w[f] > threshold ? 1 : 0;
        if (keep[f]) kept[n++] = (int32_t)f;
    }
    return n;
}
