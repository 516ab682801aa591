/* Bucket (variable) elimination of Section 3.B.1, with the slicing of Section 3.B.2.
 * TEST INFRASTRUCTURE ONLY: the CPU oracle. Plain loops, complex128, no blocking.
 *
 * A tensor is a list of variables and 2^rank complex entries; bit j of an entry's index
 * is the value of vars[j]. For each requested slice (an assignment of the sliced
 * variables, bit i of the slice number = value of slice_vars[i]):
 *   1. substitute the sliced values into every tensor (fixing a vertex, Section 3.B.2);
 *   2. for each v of the order: gather the tensors T_v that hold v, multiply them into
 *      sigma over V_v and sum sigma over v (steps 1-3 of Section 3.B.1), then replace
 *      T_v by the result (step 4);
 *   3. the remaining tensors have rank 0; their product is this slice's term.
 * Slices run in parallel with OpenMP; each writes its own output slot.
 */
#include <complex.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
#define MAXR 64

typedef struct {
    int rank;
    int vars[MAXR];
    cplx *d;
} tensor;

/* Substitute fixed values (val[v] in {0,1}, or -1 when free) into t. */
static int restrict_tensor(const tensor *t, const signed char *val, tensor *out) {
    int keep[MAXR], nk = 0;
    long fixed_mask = 0, fixed_bits = 0;
    for (int j = 0; j < t->rank; j++) {
        int v = t->vars[j];
        if (val[v] < 0) {
            keep[nk] = j;
            out->vars[nk++] = v;
        } else {
            fixed_mask |= 1L << j;
            if (val[v]) fixed_bits |= 1L << j;
        }
    }
    out->rank = nk;
    out->d = (cplx *)malloc(sizeof(cplx) << nk);
    if (!out->d) return 1;
    for (long a = 0; a < (1L << nk); a++) {
        long i = fixed_bits;
        for (int j = 0; j < nk; j++)
            if ((a >> j) & 1) i |= 1L << keep[j];
        out->d[a] = t->d[i];
    }
    (void)fixed_mask;
    return 0;
}

static int has_var(const tensor *t, int v) {
    for (int j = 0; j < t->rank; j++)
        if (t->vars[j] == v) return 1;
    return 0;
}

/* Eliminate v from the pool: returns 0, or 2 if sigma' would exceed max_rank, 1 on OOM. */
static int eliminate(tensor *pool, int *n_pool, int v, cplx *scalar, int max_rank) {
    int bucket[4096], nb = 0;
    int V[MAXR], nV = 1;
    V[0] = v;                                   /* v sits at bit 0 of sigma's index */
    for (int t = 0; t < *n_pool; t++) {
        if (!has_var(&pool[t], v)) continue;
        if (nb >= 4096) return 1;
        bucket[nb++] = t;
        for (int j = 0; j < pool[t].rank; j++) {
            int u = pool[t].vars[j], seen = 0;
            for (int k = 0; k < nV; k++) seen |= (V[k] == u);
            if (!seen) {
                if (nV >= MAXR) return 2;
                V[nV++] = u;
            }
        }
    }
    if (nb == 0) {                              /* v appears in no tensor: sum over v of 1 */
        *scalar *= 2.0;
        return 0;
    }
    int r = nV - 1;
    if (r > max_rank) return 2;
    /* pos[b][j]: bit of sigma's index holding variable j of bucket tensor b */
    int (*pos)[MAXR] = malloc(sizeof(int[MAXR]) * nb);
    tensor res;
    res.rank = r;
    for (int k = 0; k < r; k++) res.vars[k] = V[k + 1];
    res.d = (cplx *)malloc(sizeof(cplx) << r);
    if (!pos || !res.d) { free(pos); free(res.d); return 1; }
    for (int b = 0; b < nb; b++) {
        const tensor *t = &pool[bucket[b]];
        for (int j = 0; j < t->rank; j++)
            for (int k = 0; k < nV; k++)
                if (V[k] == t->vars[j]) pos[b][j] = k;
    }
    for (long a = 0; a < (1L << r); a++) {
        cplx acc = 0;
        for (int bv = 0; bv < 2; bv++) {
            long full = (a << 1) | bv;
            cplx prod = 1;
            for (int b = 0; b < nb; b++) {
                const tensor *t = &pool[bucket[b]];
                long i = 0;
                for (int j = 0; j < t->rank; j++)
                    i |= ((full >> pos[b][j]) & 1L) << j;
                prod *= t->d[i];
            }
            acc += prod;
        }
        res.d[a] = acc;
    }
    free(pos);
    /* remove the bucket (indices ascending) and append the result */
    int w = 0;
    for (int t = 0, b = 0; t < *n_pool; t++) {
        if (b < nb && bucket[b] == t) { free(pool[t].d); b++; continue; }
        pool[w++] = pool[t];
    }
    pool[w++] = res;
    *n_pool = w;
    return 0;
}

/* Returns 0 on success; 1 out of memory, 2 rank above max_rank, 3 bad order or slice
 * set, 4 a variable left uneliminated. out[2*i], out[2*i+1] = slice term (re, im). */
int oracle_ve(int n_vars, int n_tensors, const int *rank, const int *var_off, const int *vars,
              const long *data_off, const double *data, int n_order, const int *order,
              int n_slice, const int *slice_vars, long n_items, const long *slice_ids,
              double *out, int max_rank, int n_threads) {
    /* each summed variable must be either in the order or sliced, exactly once */
    int *count = calloc(n_vars > 0 ? n_vars : 1, sizeof(int));
    if (!count) return 1;
    for (int i = 0; i < n_order; i++) {
        if (order[i] < 0 || order[i] >= n_vars) { free(count); return 3; }
        count[order[i]]++;
    }
    for (int i = 0; i < n_slice; i++) {
        if (slice_vars[i] < 0 || slice_vars[i] >= n_vars) { free(count); return 3; }
        count[slice_vars[i]]++;
    }
    for (int v = 0; v < n_vars; v++)
        if (count[v] != 1) { free(count); return 3; }
    free(count);
    if (n_slice > 62) return 3;

    int status = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (long it = 0; it < n_items; it++) {
        if (status) continue;
        signed char *val = malloc(n_vars > 0 ? n_vars : 1);
        tensor *pool = malloc(sizeof(tensor) * (n_tensors + 1));
        int n_pool = 0, err = 0;
        cplx scalar = 1;
        if (!val || !pool) err = 1;
        if (!err) {
            memset(val, -1, n_vars > 0 ? n_vars : 1);
            for (int i = 0; i < n_slice; i++) val[slice_vars[i]] = (slice_ids[it] >> i) & 1;
            for (int t = 0; t < n_tensors && !err; t++) {
                tensor src;
                src.rank = rank[t];
                for (int j = 0; j < rank[t]; j++) src.vars[j] = vars[var_off[t] + j];
                src.d = (cplx *)(data + 2 * data_off[t]);
                err = restrict_tensor(&src, val, &pool[n_pool]);
                if (!err) n_pool++;
            }
            for (int i = 0; i < n_order && !err; i++)
                err = eliminate(pool, &n_pool, order[i], &scalar, max_rank);
        }
        cplx res = scalar;
        for (int t = 0; t < n_pool; t++) {
            if (!err && pool[t].rank != 0) err = 4;
            if (!err) res *= pool[t].d[0];
            free(pool[t].d);
        }
        free(pool);
        free(val);
        if (err) {
#pragma omp atomic write
            status = err;
        }
        out[2 * it] = creal(res);
        out[2 * it + 1] = cimag(res);
    }
    return status;
}
