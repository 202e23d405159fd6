/*
 * FP64 CPU baseline on all host cores (test and benchmark infrastructure only).
 *
 * The same arithmetic as oracle.c (Eq. 1, Eq. 3-8, Algorithm 1), with the Phi
 * entries grouped by voxel for DSC and by fascicle for WC so that the host cores
 * can share the work without write conflicts (the voxel- and fiber-based
 * restructurings of Sec. 4.1.2, with OpenMP standing in for the paper's
 * multi-core CPU code).  Only the benchmark's CPU legs and the tests load it; it
 * is checked against the serial oracle and shares no code with the CUDA library.
 * Entries with equal (a, v, f) may repeat: every sum below is linear in them.
 * Compile with -fopenmp -ffp-contract=off.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_omp_threads(void) { return omp_get_max_threads(); }

void oracle_omp_set_threads(int n) { omp_set_num_threads(n); }

/* Stable counting sort of entries 0..n-1 by key (0 <= key < nkeys):
 * ptr[nkeys+1] offsets, perm[n] the entries in key order. */
void oracle_omp_group(int64_t n, const int32_t* key, int64_t nkeys, int64_t* ptr, int64_t* perm) {
    memset(ptr, 0, sizeof(int64_t) * (size_t)(nkeys + 1));
    for (int64_t i = 0; i < n; ++i) ptr[key[i] + 1] += 1;
    for (int64_t k = 0; k < nkeys; ++k) ptr[k + 1] += ptr[k];
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nkeys > 0 ? nkeys : 1));
    memcpy(next, ptr, sizeof(int64_t) * (size_t)nkeys);
    for (int64_t i = 0; i < n; ++i) perm[next[key[i]]++] = i;
    free(next);
}

/* y[:,v] = Σ over the entries k of voxel v of D[:,a_k] val_k x[f_k], voxels in parallel. */
void oracle_omp_dsc(const int64_t* vptr, const int64_t* vperm, const int32_t* atom, const int32_t* fasc,
                    const double* val, int nt, const double* D, const double* x, int64_t nv, double* y) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < nv; ++v) {
        double* yv = y + (int64_t)nt * v;
        for (int t = 0; t < nt; ++t) yv[t] = 0.0;
        for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) {
            const int64_t k = vperm[q];
            const double s = val[k] * x[fasc[k]];
            const double* d = D + (int64_t)nt * atom[k];
            for (int t = 0; t < nt; ++t) yv[t] += d[t] * s;
        }
    }
}

/* g[f] = Σ over the entries k of fascicle f of val_k <D[:,a_k], r[:,v_k]>, fascicles in parallel. */
void oracle_omp_wc(const int64_t* fptr, const int64_t* fperm, const int32_t* atom, const int32_t* voxel,
                   const double* val, int nt, const double* D, const double* r, int64_t nf, double* g) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t f = 0; f < nf; ++f) {
        double acc = 0.0;
        for (int64_t q = fptr[f]; q < fptr[f + 1]; ++q) {
            const int64_t k = fperm[q];
            const double* d = D + (int64_t)nt * atom[k];
            const double* rv = r + (int64_t)nt * voxel[k];
            double dot = 0.0;
            for (int t = 0; t < nt; ++t) dot += d[t] * rv[t];
            acc += val[k] * dot;
        }
        g[f] = acc;
    }
}

static double pdot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

typedef struct {
    int64_t it;
    double alpha, obj, gg, gg0, vv, uu;
    int32_t eq, converged;
} omp_sbb_state;

/* One SBB-NNLS iteration (Eq. 5-8, Algorithm 1) in the steps and readings of
 * oracle_sbb_step, with the SpMVs and dot products on all cores.
 * work holds 2·nt·nv + 2·nf doubles. */
void oracle_omp_sbb_step(const int64_t* vptr, const int64_t* vperm, const int64_t* fptr, const int64_t* fperm,
                         const int32_t* atom, const int32_t* voxel, const int32_t* fasc, const double* val, int nt,
                         const double* D, int64_t nv, int64_t nf, const double* b, double* w, double tol,
                         int eq7_on_even, omp_sbb_state* st, double* work) {
    if (st->converged) return;
    const int64_t ny = (int64_t)nt * nv;
    double* e = work;
    double* v = work + ny;
    double* g = work + 2 * ny;
    double* u = g + nf;
    oracle_omp_dsc(vptr, vperm, atom, fasc, val, nt, D, w, nv, e);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) e[i] -= b[i];
    st->obj = 0.5 * pdot(ny, e, e);
    oracle_omp_wc(fptr, fperm, atom, voxel, val, nt, D, e, nf, g);
    for (int64_t f = 0; f < nf; ++f)
        if (w[f] == 0.0 && g[f] > 0.0) g[f] = 0.0;
    const double gg = pdot(nf, g, g);
    st->gg = gg;
    if (st->it == 0) st->gg0 = gg;
    if (gg == 0.0 || sqrt(gg) <= tol * sqrt(st->gg0)) {
        st->converged = 1;
        st->eq = 0;
        return;
    }
    oracle_omp_dsc(vptr, vperm, atom, fasc, val, nt, D, g, nv, v);
    const double vv = pdot(ny, v, v);
    st->vv = vv;
    const int even = (st->it % 2) == 0;
    const int use7 = eq7_on_even ? even : !even;
    double alpha = st->alpha;
    if (use7) {
        st->eq = 7;
        st->uu = 0.0;
        if (vv > 0.0) alpha = gg / vv;
    } else {
        st->eq = 8;
        oracle_omp_wc(fptr, fperm, atom, voxel, val, nt, D, v, nf, u);
        const double uu = pdot(nf, u, u);
        st->uu = uu;
        if (uu > 0.0) alpha = vv / uu;
    }
    st->alpha = alpha;
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < nf; ++f) {
        const double x = w[f] - alpha * g[f];
        w[f] = x > 0.0 ? x : 0.0;
    }
    st->it += 1;
}
