/*
 * qc_oracle.c -- plain, slow, obviously-correct CPU oracle for the local-energy path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The product path never calls it and
 * shares no code with it (no headers, helpers, tables or constants).
 *
 * Everything is IEEE FP64; compile with -ffp-contract=off so that no multiply-add is
 * fused.  Reductions over samples accumulate in `long double` (80-bit extended on
 * x86-64, 128-bit IEEE quad on aarch64 Linux).
 *
 * What it computes, by paper section:
 *   - Eq. 2 (Sec. II-A): the second-quantized Hamiltonian
 *         H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r,
 *     with spin orbitals interleaved (n_1a, n_1b, ..., n_Ka, n_Kb) as the occupation
 *     number vector of Sec. II-A defines them.  Reading of the integral space: the
 *     inputs are real spatial-orbital integrals h[p][q] and chemist-notation (pq|rs)
 *     over K = N/2 orbitals, and <pq|rs> = (pr|qs) d(sp,sr) d(sq,ss).
 *   - orc_h_definition: every term of Eq. 2 applied operator by operator to each ket
 *     (the definition path).
 *   - orc_slater_condon: the Slater-Condon rules (Sec. III-B item (ii), the paper's
 *     baseline), an independent derivation of the same matrix elements.
 *   - orc_eloc: Eq. 5, E_loc(n) = sum_m <n|H|m> psi(m)/psi(n), with m running over every
 *     single and double excitation of n; "sample space" mode keeps only m found in the
 *     sorted sample table (the lookup table of Sec. IV-C-4), "accurate" mode requires
 *     every m to be in the caller's table.
 *   - orc_pairwise: the same sum found by scanning every (n, m) pair of the table and
 *     keeping those that differ by one or two electrons (no enumeration).
 *   - orc_eloc_lists / orc_pairwise_lists: the same two sums, also listing every hit of a
 *     sample as phase * (table row + 1), so that connected sets and phases can be compared
 *     pair by pair; orc_eloc_lists can also return, per sample, the sum over its hits of
 *     |psi(m)/psi(n)| times the absolute integral terms of <n|H|m> (the scale of a
 *     lower-precision element's rounding error).
 *   - orc_reduce: Eq. 1, the count-weighted mean of E_loc, and its weighted variance.
 *   - orc_grad: Eq. 4, the energy gradient 2 Re < d_theta ln Psi*(n) (E_loc - <E>) >_n as
 *     a count-weighted sample average, given the rows d_theta ln Psi*(n_i).
 *
 * Sign convention: |n> = a+_{i1} a+_{i2} ... |0> with i1 < i2 < ...; hence
 * a_q |n> = (-1)^{#occupied below q} |n - q>, and a+_p |n> = (-1)^{#occupied below p} |n + p>.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint64_t w[2]; } det_t;

/* ---------------------------------------------------------------------------------
 * bit helpers (written as loops on purpose: no popcount intrinsics)
 * -------------------------------------------------------------------------------*/
static int bit_get(const det_t *d, int k) { return (int)((d->w[k >> 6] >> (k & 63)) & 1u); }
static void bit_set(det_t *d, int k) { d->w[k >> 6] |= ((uint64_t)1) << (k & 63); }
static void bit_clr(det_t *d, int k) { d->w[k >> 6] &= ~(((uint64_t)1) << (k & 63)); }

static int count_below(const det_t *d, int k) {
    int c = 0;
    for (int m = 0; m < k; ++m) c += bit_get(d, m);
    return c;
}
static int count_between(const det_t *d, int lo, int hi) { /* strictly between */
    int c = 0;
    for (int m = lo + 1; m < hi; ++m) c += bit_get(d, m);
    return c;
}
static int count_all(const det_t *d, int n_orb) {
    int c = 0;
    for (int m = 0; m < n_orb; ++m) c += bit_get(d, m);
    return c;
}
static int count_spin(const det_t *d, int n_orb, int spin) {
    int c = 0;
    for (int m = spin; m < n_orb; m += 2) c += bit_get(d, m);
    return c;
}
static int det_cmp(const det_t *a, const det_t *b) { /* unsigned 128-bit compare, hi = w[1] */
    if (a->w[1] != b->w[1]) return a->w[1] < b->w[1] ? -1 : 1;
    if (a->w[0] != b->w[0]) return a->w[0] < b->w[0] ? -1 : 1;
    return 0;
}
static int64_t det_find(const det_t *tab, int64_t n, const det_t *x) { /* binary search */
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = det_cmp(&tab[mid], x);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/* ---------------------------------------------------------------------------------
 * spin-orbital integrals from spatial ones (Eq. 2 reading, see header)
 * -------------------------------------------------------------------------------*/
typedef struct { const double *h, *eri; int K; double e_core; } ints_t;

static double h_so(const ints_t *ig, int p, int q) {
    if ((p & 1) != (q & 1)) return 0.0;
    return ig->h[(p >> 1) * ig->K + (q >> 1)];
}
static double chem(const ints_t *ig, int p, int q, int r, int s) { /* (pq|rs), spatial */
    int K = ig->K;
    return ig->eri[(((size_t)p * K + q) * K + r) * K + s];
}
/* <pq|rs> = (pr|qs) for spin orbitals */
static double phys_so(const ints_t *ig, int p, int q, int r, int s) {
    if ((p & 1) != (r & 1) || (q & 1) != (s & 1)) return 0.0;
    return chem(ig, p >> 1, r >> 1, q >> 1, s >> 1);
}
static double asym_so(const ints_t *ig, int p, int q, int r, int s) { /* <pq||rs> */
    return phys_so(ig, p, q, r, s) - phys_so(ig, p, q, s, r);
}

/* ---------------------------------------------------------------------------------
 * operator application (definition path)
 * -------------------------------------------------------------------------------*/
static int op_annihilate(det_t *d, int k, int *sign) {
    if (!bit_get(d, k)) return 0;
    if (count_below(d, k) & 1) *sign = -*sign;
    bit_clr(d, k);
    return 1;
}
static int op_create(det_t *d, int k, int *sign) {
    if (bit_get(d, k)) return 0;
    if (count_below(d, k) & 1) *sign = -*sign;
    bit_set(d, k);
    return 1;
}

static int64_t basis_find(const det_t *basis, int64_t dim, const det_t *x) {
    return det_find(basis, dim, x);
}

/* Dense H on a sorted basis by applying every term of Eq. 2 to each ket.
 * H[row * dim + col] = <basis[row]| H |basis[col]>.  Returns 0, or -1 if a term maps a
 * ket outside the basis (the basis is not closed under H). */
int orc_h_definition(const double *h, const double *eri, double e_core, int n_orb,
                     const uint64_t *basis_words, int64_t dim, double *H) {
    ints_t In = {h, eri, n_orb / 2, e_core};
    const det_t *basis = (const det_t *)basis_words;
    int N = n_orb;
    int bad = 0;
    memset(H, 0, sizeof(double) * (size_t)dim * (size_t)dim);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int64_t col = 0; col < dim; ++col) {
        const det_t ket = basis[col];
        H[col * dim + col] += e_core;
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q) {
                double c = h_so(&In, p, q);
                if (c == 0.0) continue;
                det_t z = ket; int s = 1;
                if (!op_annihilate(&z, q, &s)) continue;
                if (!op_create(&z, p, &s)) continue;
                int64_t row = basis_find(basis, dim, &z);
                if (row < 0) { bad = 1; continue; }
                H[row * dim + col] += c * (double)s;
            }
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q)
                for (int r = 0; r < N; ++r)
                    for (int t = 0; t < N; ++t) { /* t plays the role of s in Eq. 2 */
                        double c = 0.25 * asym_so(&In, p, q, r, t);
                        if (c == 0.0) continue;
                        det_t z = ket; int s = 1;
                        if (!op_annihilate(&z, r, &s)) continue;
                        if (!op_annihilate(&z, t, &s)) continue;
                        if (!op_create(&z, q, &s)) continue;
                        if (!op_create(&z, p, &s)) continue;
                        int64_t row = basis_find(basis, dim, &z);
                        if (row < 0) { bad = 1; continue; }
                        H[row * dim + col] += c * (double)s;
                    }
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------------
 * Slater-Condon rules (independent path)
 * -------------------------------------------------------------------------------*/
/* <bra|H|ket>.  *phase receives the fermionic phase of the excitation (+1/-1, or 0 when
 * the element vanishes structurally: different particle number, spin, or degree > 2).
 * For degree 1 the phase is (-1)^{#occupied strictly between hole and particle}; for
 * degree 2 it is the product of the phases of the two successive single excitations
 * i->a then j->b, with holes i<j taken from the ket and particles a<b from the bra. */
static double slater_condon(const ints_t *ig, int n_orb, const det_t *bra, const det_t *ket,
                            int *phase) {
    *phase = 0;
    if (count_all(bra, n_orb) != count_all(ket, n_orb)) return 0.0;
    if (count_spin(bra, n_orb, 0) != count_spin(ket, n_orb, 0)) return 0.0;
    int holes[2], parts[2], nh = 0, np = 0, ndiff = 0;
    for (int m = 0; m < n_orb; ++m) {
        int b = bit_get(bra, m), k = bit_get(ket, m);
        if (b != k) {
            ++ndiff;
            if (ndiff > 4) return 0.0;
            if (k) holes[nh++] = m; else parts[np++] = m;
        }
    }
    if (ndiff == 0) {
        double e = ig->e_core;
        for (int i = 0; i < n_orb; ++i) {
            if (!bit_get(ket, i)) continue;
            e += h_so(ig, i, i);
            for (int j = 0; j < n_orb; ++j)
                if (bit_get(ket, j)) e += 0.5 * asym_so(ig, i, j, i, j);
        }
        *phase = 1;
        return e;
    }
    if (ndiff == 2) {
        int i = holes[0], a = parts[0];
        int lo = i < a ? i : a, hi = i < a ? a : i;
        int ph = (count_between(ket, lo, hi) & 1) ? -1 : 1;
        double v = h_so(ig, a, i);
        for (int j = 0; j < n_orb; ++j)
            if (bit_get(ket, j)) v += asym_so(ig, a, j, i, j);
        *phase = ph;
        return (double)ph * v;
    }
    /* ndiff == 4 */
    int i = holes[0], j = holes[1], a = parts[0], b = parts[1];
    det_t mid = *ket;
    int lo = i < a ? i : a, hi = i < a ? a : i;
    int ph = (count_between(&mid, lo, hi) & 1) ? -1 : 1;
    bit_clr(&mid, i);
    bit_set(&mid, a);
    lo = j < b ? j : b; hi = j < b ? b : j;
    if (count_between(&mid, lo, hi) & 1) ph = -ph;
    *phase = ph;
    return (double)ph * asym_so(ig, a, b, i, j);
}

/* Sum of the absolute values of the integral terms that make up an off-diagonal element
 * <bra|H|ket> in the Slater-Condon rules above (no cancellation between them): for a single
 * i -> a, |h_ai| + sum over occupied j of |<aj|ij>| + |<aj|ji>|; for a double (i, j) ->
 * (a, b), |<ab|ij>| + |<ab|ji>|; 0 for the diagonal and for unconnected pairs.  It is the
 * scale of the rounding error of an element formed in a lower precision (a forward-error
 * bound of its terms' sum), not a matrix element. */
static double slater_condon_mag(const ints_t *ig, int n_orb, const det_t *bra, const det_t *ket) {
    if (count_all(bra, n_orb) != count_all(ket, n_orb)) return 0.0;
    if (count_spin(bra, n_orb, 0) != count_spin(ket, n_orb, 0)) return 0.0;
    int holes[2], parts[2], nh = 0, np = 0, ndiff = 0;
    for (int m = 0; m < n_orb; ++m) {
        int b = bit_get(bra, m), k = bit_get(ket, m);
        if (b != k) {
            ++ndiff;
            if (ndiff > 4) return 0.0;
            if (k) holes[nh++] = m; else parts[np++] = m;
        }
    }
    if (ndiff == 2) {
        int i = holes[0], a = parts[0];
        double v = fabs(h_so(ig, a, i));
        for (int j = 0; j < n_orb; ++j)
            if (bit_get(ket, j)) v += fabs(phys_so(ig, a, j, i, j)) + fabs(phys_so(ig, a, j, j, i));
        return v;
    }
    if (ndiff == 4) {
        int i = holes[0], j = holes[1], a = parts[0], b = parts[1];
        return fabs(phys_so(ig, a, b, i, j)) + fabs(phys_so(ig, a, b, j, i));
    }
    return 0.0;
}

double orc_slater_condon(const double *h, const double *eri, double e_core, int n_orb,
                         const uint64_t *bra, const uint64_t *ket, int *phase) {
    ints_t In = {h, eri, n_orb / 2, e_core};
    return slater_condon(&In, n_orb, (const det_t *)bra, (const det_t *)ket, phase);
}

int orc_h_slater_condon(const double *h, const double *eri, double e_core, int n_orb,
                        const uint64_t *basis_words, int64_t dim, double *H) {
    ints_t In = {h, eri, n_orb / 2, e_core};
    const det_t *basis = (const det_t *)basis_words;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < dim; ++r)
        for (int64_t c = 0; c < dim; ++c) {
            int ph;
            H[r * dim + c] = slater_condon(&In, n_orb, &basis[r], &basis[c], &ph);
        }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Eq. 5 by enumeration and lookup
 * -------------------------------------------------------------------------------*/
#define ORC_SAMPLE 0
#define ORC_FULL 1

typedef struct {
    const ints_t *ig; int n_orb;
    const det_t *tab; const double complex *tpsi; int64_t ntab; int mode;
    const det_t *x; double complex inv_ref; double complex psi_x;
    double complex acc; uint64_t pairs, hits, missing, rowsum; int64_t signsum;
    int64_t *list; int64_t lpos;  /* per-pair output: phase * (row + 1) of each hit, or NULL */
    int want_mag; double mag;     /* sum over hits of slater_condon_mag * |psi(x')/psi(x)| */
} eloc_ctx;

static void visit(eloc_ctx *c, const det_t *xp) {
    c->pairs++;
    int64_t row = det_find(c->tab, c->ntab, xp);
    if (row < 0) {
        if (c->mode == ORC_FULL) c->missing++;
        return;
    }
    int ph;
    double hv = slater_condon(c->ig, c->n_orb, c->x, xp, &ph);
    c->acc += hv * (c->tpsi[row] / c->psi_x);
    c->hits++;
    c->rowsum += (uint64_t)(row + 1);
    c->signsum += (int64_t)ph * (row + 1);
    if (c->list) c->list[c->lpos++] = (int64_t)ph * (row + 1);
    if (c->want_mag) c->mag += slater_condon_mag(c->ig, c->n_orb, c->x, xp) * cabs(c->tpsi[row] / c->psi_x);
}

/* For each sample x: E_loc(x) = <x|H|x> + sum over every single and double excitation
 * x' of x that conserves S_z, of <x|H|x'> psi(x')/psi(x), where psi(x') comes from the
 * table (keys sorted ascending, unique).  SAMPLE mode skips x' absent from the table;
 * FULL mode counts them as missing and sets E_loc(x) to NaN.  psi(x) == 0 gives NaN.
 * Outputs (any may be NULL except eloc): eloc complex[n_u]; per-sample pair count,
 * hit count, sum of (row+1) and sum of phase*(row+1) over hits.
 * Returns the number of samples whose E_loc is NaN. */
static int64_t eloc_enum(const double *h, const double *eri, double e_core, int n_orb,
                         const uint64_t *samples, const double *psi, int64_t n_u,
                         const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                         int mode, double *eloc, uint64_t *pairs_out, uint32_t *hits_out,
                         uint64_t *rowsum_out, int64_t *signsum_out, const int64_t *list_off,
                         int64_t *list_out, double *mag_out, int nthreads) {
    ints_t In = {h, eri, n_orb / 2, e_core};
    const det_t *S = (const det_t *)samples;
    const double complex *P = (const double complex *)psi;
    const det_t *T = table_keys ? (const det_t *)table_keys : S;
    const double complex *TP = table_keys ? (const double complex *)table_psi : P;
    int64_t NT = table_keys ? n_table : n_u;
    int64_t nbad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nbad)
    for (int64_t r = 0; r < n_u; ++r) {
        eloc_ctx c;
        memset(&c, 0, sizeof c);
        c.ig = &In; c.n_orb = n_orb; c.tab = T; c.tpsi = TP; c.ntab = NT; c.mode = mode;
        c.x = &S[r]; c.psi_x = P[r];
        if (list_off && list_out) c.list = list_out + list_off[r];
        c.want_mag = mag_out != NULL;
        const det_t x = S[r];
        int N = n_orb;
        /* singles: p occupied -> a empty, same spin */
        for (int p = 0; p < N; ++p) {
            if (!bit_get(&x, p)) continue;
            for (int a = 0; a < N; ++a) {
                if (bit_get(&x, a) || ((a & 1) != (p & 1))) continue;
                det_t y = x; bit_clr(&y, p); bit_set(&y, a);
                visit(&c, &y);
            }
        }
        /* doubles: p<q occupied -> a<b empty, spins conserved as a multiset */
        for (int p = 0; p < N; ++p) {
            if (!bit_get(&x, p)) continue;
            for (int q = p + 1; q < N; ++q) {
                if (!bit_get(&x, q)) continue;
                for (int a = 0; a < N; ++a) {
                    if (bit_get(&x, a)) continue;
                    for (int b = a + 1; b < N; ++b) {
                        if (bit_get(&x, b)) continue;
                        int sp = (p & 1) + (q & 1), sa = (a & 1) + (b & 1);
                        if (sp != sa) continue;
                        det_t y = x;
                        bit_clr(&y, p); bit_clr(&y, q); bit_set(&y, a); bit_set(&y, b);
                        visit(&c, &y);
                    }
                }
            }
        }
        int ph;
        double ed = slater_condon(&In, n_orb, &x, &x, &ph);
        double complex e = ed + c.acc;
        int isbad = (P[r] == 0.0) || (mode == ORC_FULL && c.missing > 0);
        if (isbad) { e = CMPLX(NAN, NAN); nbad++; }
        eloc[2 * r] = creal(e);
        eloc[2 * r + 1] = cimag(e);
        if (pairs_out) pairs_out[r] = c.pairs;
        if (hits_out) hits_out[r] = (uint32_t)c.hits;
        if (rowsum_out) rowsum_out[r] = c.rowsum;
        if (signsum_out) signsum_out[r] = c.signsum;
        if (mag_out) mag_out[r] = c.mag;
    }
    return nbad;
}

int64_t orc_eloc(const double *h, const double *eri, double e_core, int n_orb,
                 const uint64_t *samples, const double *psi, int64_t n_u,
                 const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                 int mode, double *eloc, uint64_t *pairs_out, uint32_t *hits_out,
                 uint64_t *rowsum_out, int64_t *signsum_out, int nthreads) {
    return eloc_enum(h, eri, e_core, n_orb, samples, psi, n_u, table_keys, table_psi, n_table, mode, eloc,
                     pairs_out, hits_out, rowsum_out, signsum_out, NULL, NULL, NULL, nthreads);
}

/* orc_eloc with two more outputs.  list_off[r] (int64, caller-computed from the hit counts
 * of a previous call) is where sample r's hits start in list_out; each hit writes
 * phase * (table row + 1) there, in the order the enumeration visits them.  mag_out[r]
 * (may be NULL) is the sum over sample r's hits of slater_condon_mag times
 * |psi(x')/psi(x)|. */
int64_t orc_eloc_lists(const double *h, const double *eri, double e_core, int n_orb,
                       const uint64_t *samples, const double *psi, int64_t n_u,
                       const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                       int mode, double *eloc, const int64_t *list_off, int64_t *list_out,
                       double *mag_out, int nthreads) {
    return eloc_enum(h, eri, e_core, n_orb, samples, psi, n_u, table_keys, table_psi, n_table, mode, eloc,
                     NULL, NULL, NULL, NULL, list_off, list_out, mag_out, nthreads);
}

/* Same sum by an O(n_u * n_table) scan: y is connected to x when they hold the same
 * number of alpha and of beta electrons and differ in exactly 2 or 4 spin orbitals. */
static int64_t pairwise_scan(const double *h, const double *eri, double e_core, int n_orb,
                             const uint64_t *samples, const double *psi, int64_t n_u,
                             const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                             double *eloc, uint32_t *hits_out, uint64_t *rowsum_out,
                             int64_t *signsum_out, const int64_t *list_off, int64_t *list_out,
                             int nthreads) {
    ints_t In = {h, eri, n_orb / 2, e_core};
    const det_t *S = (const det_t *)samples;
    const double complex *P = (const double complex *)psi;
    const det_t *T = table_keys ? (const det_t *)table_keys : S;
    const double complex *TP = table_keys ? (const double complex *)table_psi : P;
    int64_t NT = table_keys ? n_table : n_u;
    int64_t nbad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nbad)
    for (int64_t r = 0; r < n_u; ++r) {
        const det_t x = S[r];
        int na = count_spin(&x, n_orb, 0), nb = count_spin(&x, n_orb, 1);
        double complex acc = 0;
        uint64_t hits = 0, rs = 0; int64_t ss = 0;
        for (int64_t t = 0; t < NT; ++t) {
            const det_t *y = &T[t];
            int diff = 0;
            for (int m = 0; m < n_orb; ++m) diff += bit_get(&x, m) != bit_get(y, m);
            if (diff != 2 && diff != 4) continue;
            if (count_spin(y, n_orb, 0) != na || count_spin(y, n_orb, 1) != nb) continue;
            int ph;
            double hv = slater_condon(&In, n_orb, &x, y, &ph);
            acc += hv * (TP[t] / P[r]);
            if (list_off && list_out) list_out[list_off[r] + (int64_t)hits] = (int64_t)ph * (t + 1);
            hits++; rs += (uint64_t)(t + 1); ss += (int64_t)ph * (t + 1);
        }
        int ph;
        double complex e = slater_condon(&In, n_orb, &x, &x, &ph) + acc;
        if (P[r] == 0.0) { e = CMPLX(NAN, NAN); nbad++; }
        eloc[2 * r] = creal(e);
        eloc[2 * r + 1] = cimag(e);
        if (hits_out) hits_out[r] = (uint32_t)hits;
        if (rowsum_out) rowsum_out[r] = rs;
        if (signsum_out) signsum_out[r] = ss;
    }
    return nbad;
}

int64_t orc_pairwise(const double *h, const double *eri, double e_core, int n_orb,
                     const uint64_t *samples, const double *psi, int64_t n_u,
                     const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                     double *eloc, uint32_t *hits_out, uint64_t *rowsum_out,
                     int64_t *signsum_out, int nthreads) {
    return pairwise_scan(h, eri, e_core, n_orb, samples, psi, n_u, table_keys, table_psi, n_table, eloc,
                         hits_out, rowsum_out, signsum_out, NULL, NULL, nthreads);
}

/* orc_pairwise writing each sample's hits as phase * (table row + 1) from list_off[r] on,
 * in table order. */
int64_t orc_pairwise_lists(const double *h, const double *eri, double e_core, int n_orb,
                           const uint64_t *samples, const double *psi, int64_t n_u,
                           const uint64_t *table_keys, const double *table_psi, int64_t n_table,
                           double *eloc, const int64_t *list_off, int64_t *list_out, int nthreads) {
    return pairwise_scan(h, eri, e_core, n_orb, samples, psi, n_u, table_keys, table_psi, n_table, eloc,
                         NULL, NULL, NULL, list_off, list_out, nthreads);
}

/* ---------------------------------------------------------------------------------
 * Eq. 1 reduction
 * -------------------------------------------------------------------------------*/
/* out[0..4] = { Re Ebar, Im Ebar, var, W, n_used }:
 *   W = sum c_i,  Ebar = sum c_i E_i / W,  var = sum c_i |E_i - Ebar|^2 / W
 * over samples whose E_loc is finite (two passes, long double accumulators). */
int orc_reduce(const double *eloc, const int64_t *counts, int64_t n, double *out) {
    long double w = 0, sr = 0, si = 0;
    int64_t used = 0;
    for (int64_t i = 0; i < n; ++i) {
        double er = eloc[2 * i], ei = eloc[2 * i + 1];
        if (!isfinite(er) || !isfinite(ei)) continue;
        long double c = (long double)counts[i];
        w += c; sr += c * er; si += c * ei; used++;
    }
    long double mr = sr / w, mi = si / w, v = 0;
    for (int64_t i = 0; i < n; ++i) {
        double er = eloc[2 * i], ei = eloc[2 * i + 1];
        if (!isfinite(er) || !isfinite(ei)) continue;
        long double dr = er - mr, di = ei - mi;
        v += (long double)counts[i] * (dr * dr + di * di);
    }
    out[0] = (double)mr; out[1] = (double)mi; out[2] = (double)(v / w);
    out[3] = (double)w; out[4] = (double)used;
    return 0;
}

/* Eq. 4 over the unique samples: with W = sum c_i and Ebar the Eq. 1 mean (complex),
 *   w_i = c_i (E_loc,i - Ebar) / W      (0 for a sample whose E_loc is not finite)
 *   g_p = 2 Re sum_i w_i D_ip,          D_ip = d/d theta_p ln Psi*(n_i)  (complex, row-major)
 * Written as two plain loops in long double.  w_out (complex, n) or g_out (P) may be NULL. */
int orc_grad(const double *eloc, const int64_t *counts, int64_t n, const double *dconj, int64_t P,
             double *w_out, double *g_out) {
    long double W = 0, sr = 0, si = 0;
    for (int64_t i = 0; i < n; ++i) {
        double er = eloc[2 * i], ei = eloc[2 * i + 1];
        if (!isfinite(er) || !isfinite(ei)) continue;
        W += (long double)counts[i];
        sr += (long double)counts[i] * er;
        si += (long double)counts[i] * ei;
    }
    if (W <= 0) return -1;
    const long double mr = sr / W, mi = si / W;
    long double *wr = (long double *)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
    long double *wi = (long double *)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
    if (!wr || !wi) { free(wr); free(wi); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        double er = eloc[2 * i], ei = eloc[2 * i + 1];
        if (!isfinite(er) || !isfinite(ei)) continue;
        wr[i] = (long double)counts[i] * (er - mr) / W;
        wi[i] = (long double)counts[i] * (ei - mi) / W;
    }
    if (w_out)
        for (int64_t i = 0; i < n; ++i) { w_out[2 * i] = (double)wr[i]; w_out[2 * i + 1] = (double)wi[i]; }
    if (g_out && dconj)
        for (int64_t p = 0; p < P; ++p) {
            long double g = 0;
            for (int64_t i = 0; i < n; ++i) {
                const double dr = dconj[2 * (i * P + p)], di = dconj[2 * (i * P + p) + 1];
                g += wr[i] * dr - wi[i] * di;   /* Re(w D) */
            }
            g_out[p] = (double)(2 * g);
        }
    free(wr);
    free(wi);
    return 0;
}

/* Every S_z-conserving single and double excitation of each sample, deduplicated and
 * sorted: a table that covers the whole connected set ("accurate" mode input). */
static int cmp_det(const void *a, const void *b) { return det_cmp((const det_t *)a, (const det_t *)b); }

int64_t orc_connected_union(int n_orb, const uint64_t *samples, int64_t n_u,
                            uint64_t *out_words, int64_t cap) {
    const det_t *S = (const det_t *)samples;
    det_t *out = (det_t *)out_words;
    int64_t n = 0;
    int N = n_orb;
    for (int64_t r = 0; r < n_u; ++r) {
        const det_t x = S[r];
        for (int p = 0; p < N; ++p) {
            if (!bit_get(&x, p)) continue;
            for (int a = 0; a < N; ++a) {
                if (bit_get(&x, a) || ((a & 1) != (p & 1))) continue;
                if (n >= cap) return -1;
                det_t y = x; bit_clr(&y, p); bit_set(&y, a); out[n++] = y;
            }
            for (int q = p + 1; q < N; ++q) {
                if (!bit_get(&x, q)) continue;
                for (int a = 0; a < N; ++a) {
                    if (bit_get(&x, a)) continue;
                    for (int b = a + 1; b < N; ++b) {
                        if (bit_get(&x, b)) continue;
                        if ((p & 1) + (q & 1) != (a & 1) + (b & 1)) continue;
                        if (n >= cap) return -1;
                        det_t y = x;
                        bit_clr(&y, p); bit_clr(&y, q); bit_set(&y, a); bit_set(&y, b);
                        out[n++] = y;
                    }
                }
            }
        }
    }
    qsort(out, (size_t)n, sizeof(det_t), cmp_det);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || det_cmp(&out[m - 1], &out[i]) != 0) out[m++] = out[i];
    return m;
}

/* Every bitstring with n_alpha alpha and n_beta beta electrons, sorted. */
int64_t orc_sector(int n_orb, int n_alpha, int n_beta, uint64_t *out_words, int64_t cap) {
    det_t *out = (det_t *)out_words;
    int64_t n = 0;
    int K = n_orb / 2;
    if (K > 20) return -1; /* brute force only */
    for (uint64_t a = 0; a < (1ull << K); ++a) {
        int ca = 0;
        for (int k = 0; k < K; ++k) ca += (int)((a >> k) & 1);
        if (ca != n_alpha) continue;
        for (uint64_t b = 0; b < (1ull << K); ++b) {
            int cb = 0;
            for (int k = 0; k < K; ++k) cb += (int)((b >> k) & 1);
            if (cb != n_beta) continue;
            det_t d = {{0, 0}};
            for (int k = 0; k < K; ++k) {
                if ((a >> k) & 1) bit_set(&d, 2 * k);
                if ((b >> k) & 1) bit_set(&d, 2 * k + 1);
            }
            if (n >= cap) return -1;
            out[n++] = d;
        }
    }
    qsort(out, (size_t)n, sizeof(det_t), cmp_det);
    return n;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
