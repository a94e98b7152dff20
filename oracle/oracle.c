/*
 * Plain FP64 CPU oracle for the deterministic NQS hot path (arXiv 2601.21310).
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into oracle/liboracle.so and is loaded only
 * by the tests, by the package smoke check and by the benchmark's CPU-baseline leg. It shares
 * no code, header or table with the CUDA library; the two meet only through the seeded inputs.
 *
 * Everything here is written to be checked by eye against the paper:
 *   - the Hamiltonian is the usual second-quantised electronic Hamiltonian in the Fock basis of
 *     Sec. 2.1; its matrix elements between configurations follow the Slater-Condon rules that
 *     Sec. 3.1 names for the combinatorial kernel (the rules themselves are textbook);
 *   - the connected set is Eq. (connected_set) (all singles and doubles of each x in S);
 *   - the ansatz is Eqs. (effective_orbital_matrix), (occupied_submatrix), (backflow_amplitude)
 *     in the spin-blocked form psi = det Phi[occ_a, 0:na] * det Phi[occ_b, na:na+nb];
 *   - the objective and its gradient are Eqs. (variational_energy), (variational_gradient);
 *   - the perturbative correction is Eq. (pt2_correction);
 *   - the heat-bath screened perturbative set is Eq. (hb_screen);
 *   - the subspace selector of the outer loop is Sec. 2.4.2 (Top-K, cumulative mass,
 *     absolute threshold);
 *   - the Proxy-mode Hamiltonian is Eq. (proxy_hamiltonian); the Asymmetric mode is
 *     Eqs. (asymmetric_energy), (asymmetric_gradient) with its exact gradient derived here.
 *
 * Conventions fixed here (the paper is silent on them):
 *   - spin-orbital order alpha 0..norb-1, then beta 0..norb-1; |x> = prod over occupied
 *     spin-orbitals in ascending order of creation operators acting on |0>;
 *   - a configuration is the word pair (a, b); bit p of a (b) = alpha (beta) orbital p occupied;
 *   - ERIs in chemists' notation (pq|rs), eri[((p*norb+q)*norb+r)*norb+s];
 *   - canonical excitation order of one configuration: alpha singles (i asc, a asc), beta
 *     singles, alpha-alpha doubles (i<j pairs lexicographic, then a<b pairs lexicographic),
 *     beta-beta doubles, alpha-beta doubles (i_a asc, a_a asc, j_b asc, b_b asc);
 *   - a CSR row of H_SS is [diagonal, then the hits of the canonical excitation list in order].
 *
 * No fused multiply-add: compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_OOM -5
#define ORC_WARN_SINGULAR 1

static inline int popc(uint64_t v) { return __builtin_popcountll(v); }

/* occupied orbitals of a word, ascending; returns count */
static int occ_list(uint64_t w, int norb, int* out) {
    int n = 0;
    for (int p = 0; p < norb; ++p)
        if ((w >> p) & 1ull) out[n++] = p;
    return n;
}
static int vir_list(uint64_t w, int norb, int* out) {
    int n = 0;
    for (int p = 0; p < norb; ++p)
        if (!((w >> p) & 1ull)) out[n++] = p;
    return n;
}

/* bits strictly between orbitals p and q */
static inline uint64_t between(int p, int q) {
    int lo = p < q ? p : q, hi = p < q ? q : p;
    uint64_t below_hi = (hi >= 64) ? ~0ull : ((1ull << hi) - 1ull);
    uint64_t upto_lo = (lo + 1 >= 64) ? ~0ull : ((1ull << (lo + 1)) - 1ull);
    return below_hi & ~upto_lo;
}

/* sign of a^dagger_a a_i on one spin string w (i occupied, a empty): (-1)^(# occupied strictly
 * between i and a). The other spin string contributes an even count and drops out. */
static inline int single_sign(uint64_t w, int i, int a) {
    return (popc(w & between(i, a)) & 1) ? -1 : 1;
}

#define ERI(p, q, r, s) eri[(((size_t)(p) * norb + (q)) * norb + (r)) * norb + (s)]

/* ------------------------------------------------------------------------------------------
 * Diagonal element (Slater-Condon, zero excitations):
 *   H_xx = sum_{i in occ_a} h_ii + sum_{i in occ_b} h_ii
 *        + sum_{i<j in occ_a} [(ii|jj) - (ij|ji)] + same for beta
 *        + sum_{i in occ_a, j in occ_b} (ii|jj).
 * Accumulated in exactly that order into one running sum. ecore is not included.
 * ---------------------------------------------------------------------------------------- */
double orc_diag(int norb, const double* h, const double* eri, uint64_t a, uint64_t b) {
    int oa[64], ob[64];
    int na = occ_list(a, norb, oa), nb = occ_list(b, norb, ob);
    double e = 0.0;
    for (int k = 0; k < na; ++k) e = e + h[oa[k] * norb + oa[k]];
    for (int k = 0; k < nb; ++k) e = e + h[ob[k] * norb + ob[k]];
    for (int x = 0; x < na; ++x)
        for (int y = x + 1; y < na; ++y) {
            int i = oa[x], j = oa[y];
            double t = ERI(i, i, j, j) - ERI(i, j, j, i);
            e = e + t;
        }
    for (int x = 0; x < nb; ++x)
        for (int y = x + 1; y < nb; ++y) {
            int i = ob[x], j = ob[y];
            double t = ERI(i, i, j, j) - ERI(i, j, j, i);
            e = e + t;
        }
    for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) {
            int i = oa[x], j = ob[y];
            e = e + ERI(i, i, j, j);
        }
    return e;
}

/* ------------------------------------------------------------------------------------------
 * General matrix element <y|H|x> between two configurations of the same sector.
 * Returns the excitation level (0, 1, 2) in *level, or 3 when they differ by more than a
 * double (element 0).
 *   single i->a in spin s: sign * [ h_ia + sum_{j in occ_a(x)&occ_a(y), asc} t_a(j)
 *                                        + sum_{j in occ_b(x)&occ_b(y), asc} t_b(j) ]
 *       with t(j) = (ia|jj) - (ij|ja) for j of spin s and t(j) = (ia|jj) otherwise;
 *   same-spin double i<j -> a<b: s(i->a on x) * s(j->b after it) * [(ia|jb) - (ib|ja)];
 *   opposite-spin double i->a (alpha), j->b (beta): s_a * s_b * (ia|jb).
 * ---------------------------------------------------------------------------------------- */
double orc_element(int norb, const double* h, const double* eri, uint64_t xa, uint64_t xb,
                   uint64_t ya, uint64_t yb, int* level) {
    int da = popc(xa ^ ya) / 2, db = popc(xb ^ yb) / 2;
    int lv = da + db;
    if (level) *level = lv > 2 ? 3 : lv;
    if (lv == 0) return orc_diag(norb, h, eri, xa, xb);
    if (lv > 2) return 0.0;
    if (lv == 1) {
        int spin = da == 1 ? 0 : 1;
        uint64_t xs = spin == 0 ? xa : xb, ys = spin == 0 ? ya : yb;
        int i = __builtin_ctzll(xs & ~ys), a = __builtin_ctzll(ys & ~xs);
        int sg = single_sign(xs, i, a);
        double v = h[i * norb + a];
        uint64_t ca = xa & ya, cb = xb & yb;
        for (int j = 0; j < norb; ++j) {
            if (!((ca >> j) & 1ull)) continue;
            if (spin == 0) {
                double t = ERI(i, a, j, j) - ERI(i, j, j, a);
                v = v + t;
            } else {
                v = v + ERI(i, a, j, j);
            }
        }
        for (int j = 0; j < norb; ++j) {
            if (!((cb >> j) & 1ull)) continue;
            if (spin == 1) {
                double t = ERI(i, a, j, j) - ERI(i, j, j, a);
                v = v + t;
            } else {
                v = v + ERI(i, a, j, j);
            }
        }
        return sg < 0 ? -v : v;
    }
    /* doubles */
    if (da == 2 || db == 2) {
        uint64_t xs = da == 2 ? xa : xb, ys = da == 2 ? ya : yb;
        uint64_t hole = xs & ~ys, part = ys & ~xs;
        int i = __builtin_ctzll(hole), j = 63 - __builtin_clzll(hole);
        int a = __builtin_ctzll(part), b = 63 - __builtin_clzll(part);
        int s1 = single_sign(xs, i, a);
        uint64_t x1 = xs ^ (1ull << i) ^ (1ull << a);
        int s2 = single_sign(x1, j, b);
        double t = ERI(i, a, j, b) - ERI(i, b, j, a);
        return (s1 * s2) < 0 ? -t : t;
    }
    {
        int i = __builtin_ctzll(xa & ~ya), a = __builtin_ctzll(ya & ~xa);
        int j = __builtin_ctzll(xb & ~yb), b = __builtin_ctzll(yb & ~xb);
        int sg = single_sign(xa, i, a) * single_sign(xb, j, b);
        double t = ERI(i, a, j, b);
        return sg < 0 ? -t : t;
    }
}

/* ------------------------------------------------------------------------------------------
 * Connected set of one configuration, Eq. (connected_set): every single and double
 * excitation, in the canonical order stated at the top of this file.
 * ---------------------------------------------------------------------------------------- */
int64_t orc_n_excitations(int norb, int na, int nb) {
    int64_t ma = norb - na, mb = norb - nb;
    int64_t sa = (int64_t)na * ma, sb = (int64_t)nb * mb;
    int64_t daa = (int64_t)na * (na - 1) / 2 * (ma * (ma - 1) / 2);
    int64_t dbb = (int64_t)nb * (nb - 1) / 2 * (mb * (mb - 1) / 2);
    return sa + sb + daa + dbb + sa * sb;
}

int64_t orc_excitations(int norb, uint64_t a, uint64_t b, uint64_t* out) {
    int oa[64], va[64], ob[64], vb[64];
    int na = occ_list(a, norb, oa), ma = vir_list(a, norb, va);
    int nb = occ_list(b, norb, ob), mb = vir_list(b, norb, vb);
    int64_t k = 0;
    for (int x = 0; x < na; ++x)
        for (int y = 0; y < ma; ++y) {
            out[2 * k] = a ^ (1ull << oa[x]) ^ (1ull << va[y]);
            out[2 * k + 1] = b;
            ++k;
        }
    for (int x = 0; x < nb; ++x)
        for (int y = 0; y < mb; ++y) {
            out[2 * k] = a;
            out[2 * k + 1] = b ^ (1ull << ob[x]) ^ (1ull << vb[y]);
            ++k;
        }
    for (int x1 = 0; x1 < na; ++x1)
        for (int x2 = x1 + 1; x2 < na; ++x2)
            for (int y1 = 0; y1 < ma; ++y1)
                for (int y2 = y1 + 1; y2 < ma; ++y2) {
                    out[2 * k] = a ^ (1ull << oa[x1]) ^ (1ull << oa[x2]) ^ (1ull << va[y1]) ^
                                 (1ull << va[y2]);
                    out[2 * k + 1] = b;
                    ++k;
                }
    for (int x1 = 0; x1 < nb; ++x1)
        for (int x2 = x1 + 1; x2 < nb; ++x2)
            for (int y1 = 0; y1 < mb; ++y1)
                for (int y2 = y1 + 1; y2 < mb; ++y2) {
                    out[2 * k] = a;
                    out[2 * k + 1] = b ^ (1ull << ob[x1]) ^ (1ull << ob[x2]) ^ (1ull << vb[y1]) ^
                                     (1ull << vb[y2]);
                    ++k;
                }
    for (int x = 0; x < na; ++x)
        for (int y = 0; y < ma; ++y)
            for (int u = 0; u < nb; ++u)
                for (int w = 0; w < mb; ++w) {
                    out[2 * k] = a ^ (1ull << oa[x]) ^ (1ull << va[y]);
                    out[2 * k + 1] = b ^ (1ull << ob[u]) ^ (1ull << vb[w]);
                    ++k;
                }
    return k;
}

/* position of (a, b) in the key-sorted set S, or -1 */
static int64_t find_in_S(const uint64_t* S, int64_t nS, uint64_t a, uint64_t b) {
    int64_t lo = 0, hi = nS - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        uint64_t ma = S[2 * mid], mb = S[2 * mid + 1];
        if (ma == a && mb == b) return mid;
        if (ma < a || (ma == a && mb < b)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------------
 * H_SS in CSR (Sec. 3.1: the combinatorial kernel exports H_VV as CSR).
 * Pass 1 (fill == 0) writes row lengths into row_ptr[1..nS] and the prefix sums into row_ptr.
 * Pass 2 (fill == 1) writes col/val. n_enum receives the number of (x, excitation) pairs.
 * ---------------------------------------------------------------------------------------- */
int orc_hss_rows(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                 int64_t r0, int64_t r1, int fill, int64_t* row_ptr, int32_t* col, double* val);

int orc_hss(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
            int fill, int64_t* row_ptr, int32_t* col, double* val, int64_t* n_enum) {
    if (norb < 1 || norb > 64 || nS < 0) return ORC_ERR_ARG;
    int na = popc(nS ? S[0] : 0), nb = popc(nS ? S[1] : 0);
    if (n_enum) *n_enum = orc_n_excitations(norb, na, nb) * nS;
    return orc_hss_rows(norb, h, eri, S, nS, 0, nS, fill, row_ptr, col, val);
}

/* Rows r0..r1-1 of the same CSR (lookups still into all of S); row_ptr has r1 - r0 + 1
 * entries and starts at 0. Used to check large problems on a sample of rows. */
int orc_hss_rows(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                 int64_t r0, int64_t r1, int fill, int64_t* row_ptr, int32_t* col, double* val) {
    if (norb < 1 || norb > 64 || nS < 0 || r0 < 0 || r1 > nS || r0 > r1) return ORC_ERR_ARG;
    int na = popc(nS ? S[0] : 0), nb = popc(nS ? S[1] : 0);
    int64_t nexc = orc_n_excitations(norb, na, nb);
    int err = 0;
#pragma omp parallel
    {
        uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)(nexc > 0 ? nexc : 1));
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = r0; r < r1; ++r) {
            if (!buf) continue;
            uint64_t a = S[2 * r], b = S[2 * r + 1];
            int64_t n = orc_excitations(norb, a, b, buf);
            if (!fill) {
                int64_t cnt = 1;
                for (int64_t k = 0; k < n; ++k)
                    if (find_in_S(S, nS, buf[2 * k], buf[2 * k + 1]) >= 0) ++cnt;
                row_ptr[r - r0 + 1] = cnt;
            } else {
                int64_t pos = row_ptr[r - r0];
                col[pos] = (int32_t)r;
                val[pos] = orc_diag(norb, h, eri, a, b);
                ++pos;
                for (int64_t k = 0; k < n; ++k) {
                    int64_t c = find_in_S(S, nS, buf[2 * k], buf[2 * k + 1]);
                    if (c < 0) continue;
                    col[pos] = (int32_t)c;
                    val[pos] = orc_element(norb, h, eri, a, b, buf[2 * k], buf[2 * k + 1], NULL);
                    ++pos;
                }
            }
        }
        free(buf);
    }
    if (err) return ORC_ERR_OOM;
    if (!fill) {
        row_ptr[0] = 0;
        for (int64_t r = 0; r < r1 - r0; ++r) row_ptr[r + 1] += row_ptr[r];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Compensated (Neumaier) summation, used for every long FP64 sum below.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    double s, c;
} ksum;
static inline void kadd(ksum* k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static inline double kval(const ksum* k) { return k->s + k->c; }

/* ------------------------------------------------------------------------------------------
 * BF16 rounding, from the IEEE-754 definition of round-to-nearest-even applied to the
 * binary32 bit pattern (keep the top 16 bits). Used only in the quantisation-matched mode.
 * ---------------------------------------------------------------------------------------- */
double orc_bf16_round(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan untouched */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}
static inline double f32r(double x) { return (double)(float)x; }

/* ------------------------------------------------------------------------------------------
 * Backflow network (Sec. 2.2, Sec. 3.3): MLP with two tanh hidden layers on the 0/1 input
 * (alpha bits then beta bits), linear output reshaped row-major to [norb][na+nb], added to
 * Phi0 (Eq. effective_orbital_matrix).
 * quant == 1 reproduces the mixed-precision form's rounding points: weights rounded to BF16,
 * biases and Phi0 to FP32, each hidden activation rounded to BF16 before it enters the next
 * layer; all products and sums stay FP64.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int norb, na, nb, H1, H2, quant;
    const double *W1, *b1, *W2, *b2, *W3, *b3, *Phi0;
} orc_net;

static double wq(const orc_net* n, double w) { return n->quant ? orc_bf16_round(w) : w; }
static double bq(const orc_net* n, double b) { return n->quant ? f32r(b) : b; }
static double aq(const orc_net* n, double h) { return n->quant ? orc_bf16_round(h) : h; }

/* x[2norb] input bits; h1, h2 receive the (rounded, in quant mode) activations; phi out */
static void net_forward(const orc_net* n, uint64_t a, uint64_t b, double* x, double* h1,
                        double* h2, double* phi) {
    int nin = 2 * n->norb, nel = n->na + n->nb, nout = n->norb * nel;
    for (int p = 0; p < n->norb; ++p) {
        x[p] = (double)((a >> p) & 1ull);
        x[n->norb + p] = (double)((b >> p) & 1ull);
    }
    for (int i = 0; i < n->H1; ++i) {
        double z = 0.0;
        for (int k = 0; k < nin; ++k) z += wq(n, n->W1[(size_t)i * nin + k]) * x[k];
        z += bq(n, n->b1[i]);
        h1[i] = aq(n, tanh(z));
    }
    for (int i = 0; i < n->H2; ++i) {
        double z = 0.0;
        for (int k = 0; k < n->H1; ++k) z += wq(n, n->W2[(size_t)i * n->H1 + k]) * h1[k];
        z += bq(n, n->b2[i]);
        h2[i] = aq(n, tanh(z));
    }
    for (int o = 0; o < nout; ++o) {
        double z = 0.0;
        for (int k = 0; k < n->H2; ++k) z += wq(n, n->W3[(size_t)o * n->H2 + k]) * h2[k];
        z += bq(n, n->b3[o]);
        phi[o] = bq(n, n->Phi0[o]) + z;
    }
}

/* LU with partial pivoting (Doolittle), ties broken toward the lowest row index.
 * A is n x n row-major, overwritten by L\U; perm[k] = original row now at position k.
 * Returns the sign of det (0 if a pivot is exactly zero) and log|det| in *logabs. */
static int lu_factor(double* A, int n, int* perm, double* logabs) {
    int sgn = 1;
    double la = 0.0;
    for (int k = 0; k < n; ++k) perm[k] = k;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) {
                best = fabs(A[i * n + k]);
                p = i;
            }
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
            int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
            sgn = -sgn;
        }
        double piv = A[k * n + k];
        if (piv == 0.0) {
            *logabs = -INFINITY;
            return 0;
        }
        if (piv < 0) sgn = -sgn;
        la += log(fabs(piv));
        for (int i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / piv;
            A[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    *logabs = la;
    return sgn;
}

/* inverse from the LU factors: solve A X = I column by column */
static void lu_inverse(const double* LU, const int* perm, int n, double* inv) {
    double col[64];
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) col[i] = (perm[i] == c) ? 1.0 : 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) col[i] -= LU[i * n + j] * col[j];
        for (int i = n - 1; i >= 0; --i) {
            for (int j = i + 1; j < n; ++j) col[i] -= LU[i * n + j] * col[j];
            col[i] /= LU[i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[i * n + c] = col[i];
    }
}

/* occupied submatrix of one spin block (Eq. occupied_submatrix, spin-blocked) */
static void gather_block(const double* phi, int nel, const int* occ, int n, int col0, double* A) {
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) A[j * n + k] = phi[(size_t)occ[j] * nel + col0 + k];
}

/* psi(x) = det A_a * det A_b (Eq. backflow_amplitude), as (log|psi|, sign). */
int orc_amplitudes(const orc_net* n, const uint64_t* S, int64_t nS, double* logabs, int8_t* sign) {
    int nel = n->na + n->nb;
    int status = ORC_OK;
#pragma omp parallel
    {
        double* x = (double*)malloc(sizeof(double) * 2 * n->norb);
        double* h1 = (double*)malloc(sizeof(double) * n->H1);
        double* h2 = (double*)malloc(sizeof(double) * n->H2);
        double* phi = (double*)malloc(sizeof(double) * n->norb * nel);
        double A[64 * 64];
        int perm[64], oa[64], ob[64];
#pragma omp for schedule(static)
        for (int64_t r = 0; r < nS; ++r) {
            net_forward(n, S[2 * r], S[2 * r + 1], x, h1, h2, phi);
            occ_list(S[2 * r], n->norb, oa);
            occ_list(S[2 * r + 1], n->norb, ob);
            double la, lb;
            gather_block(phi, nel, oa, n->na, 0, A);
            int sa = lu_factor(A, n->na, perm, &la);
            gather_block(phi, nel, ob, n->nb, n->na, A);
            int sb = lu_factor(A, n->nb, perm, &lb);
            logabs[r] = la + lb;
            sign[r] = (int8_t)(sa * sb);
            if (sa * sb == 0) {
#pragma omp atomic write
                status = ORC_WARN_SINGULAR;
            }
        }
        free(x);
        free(h1);
        free(h2);
        free(phi);
    }
    return status;
}

/* v = H_SS psi, row sums in CSR order */
static void spmv(const int64_t* row_ptr, const int32_t* col, const double* val, const double* psi,
                 int64_t nS, double* v) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nS; ++r) {
        double s = 0.0;
        for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) s += val[k] * psi[col[k]];
        v[r] = s;
    }
}

/* Rayleigh quotient on S for a given psi (Eq. variational_energy):
 * out = [E, N, D] with N = psi^T H_SS psi, D = psi^T psi (compensated sums in S order). */
int orc_energy_from_psi(const int64_t* row_ptr, const int32_t* col, const double* val,
                        const double* psi, int64_t nS, double* out, double* v_out) {
    double* v = v_out ? v_out : (double*)malloc(sizeof(double) * (nS > 0 ? nS : 1));
    if (!v) return ORC_ERR_OOM;
    spmv(row_ptr, col, val, psi, nS, v);
    ksum N = {0, 0}, D = {0, 0};
    for (int64_t r = 0; r < nS; ++r) {
        kadd(&N, psi[r] * v[r]);
        kadd(&D, psi[r] * psi[r]);
    }
    out[1] = kval(&N);
    out[2] = kval(&D);
    out[0] = out[1] / out[2];
    if (!v_out) free(v);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * E_S and its gradient (Eqs. variational_energy, variational_gradient).
 *   psi~_x = sign_x exp(log|psi_x| - max log|psi|)   (a global scale; E is scale invariant)
 *   v = H_SS psi~, N = psi~^T v, D = psi~^T psi~, E = N / D
 *   dE/dtheta = (2/D) sum_x (v_x - E psi~_x) dpsi~_x/dtheta
 *   dpsi~_x/dA_s = psi~_x A_s^{-T}  (Jacobi's formula), so
 *   dPhi(x)[occ_s[j], col0_s + k] = w_x (A_s^{-1})[k][j],  w_x = (2/D)(v_x - E psi~_x) psi~_x,
 *   then the chain rule through the MLP (hand-written backward, FP64).
 * out = [E, N, D, max log|psi|]; grad (may be NULL) laid out as W1, b1, W2, b2, W3, b3.
 * psi_out/v_out (may be NULL) receive psi~ and v.
 * ---------------------------------------------------------------------------------------- */
int64_t orc_n_params(const orc_net* n) {
    int nin = 2 * n->norb, nout = n->norb * (n->na + n->nb);
    return (int64_t)n->H1 * nin + n->H1 + (int64_t)n->H2 * n->H1 + n->H2 + (int64_t)nout * n->H2 +
           nout;
}

/* sum over r of coef_r * (d psi_r / d theta), with d psi / d Phi = psi A^{-T} per spin block
 * (Jacobi's formula through the LU inverse) pushed back through the MLP; written as
 * coef_r psi_r d log|psi_r| / d theta. Configurations with a singular block are skipped. */
static int grad_core(const orc_net* n, const uint64_t* S, int64_t nS, const int8_t* sg,
                     const double* psi, const double* coef, double* grad) {
    int norb = n->norb, nin = 2 * norb, nel = n->na + n->nb, nout = norb * nel;
    int64_t np = orc_n_params(n);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double* acc = (double*)calloc((size_t)np * nthr, sizeof(double));
    if (!acc) return ORC_ERR_OOM;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* g = acc + (size_t)np * tid;
        double *gW1 = g, *gb1 = gW1 + (size_t)n->H1 * nin, *gW2 = gb1 + n->H1;
        double *gb2 = gW2 + (size_t)n->H2 * n->H1, *gW3 = gb2 + n->H2;
        double* gb3 = gW3 + (size_t)nout * n->H2;
        double* x = (double*)malloc(sizeof(double) * nin);
        double* h1 = (double*)malloc(sizeof(double) * n->H1);
        double* h2 = (double*)malloc(sizeof(double) * n->H2);
        double* phi = (double*)malloc(sizeof(double) * nout);
        double* dphi = (double*)malloc(sizeof(double) * nout);
        double* dh2 = (double*)malloc(sizeof(double) * n->H2);
        double* dh1 = (double*)malloc(sizeof(double) * n->H1);
        double A[64 * 64], inv[64 * 64];
        int perm[64], oa[64], ob[64];
#pragma omp for schedule(static)
        for (int64_t r = 0; r < nS; ++r) {
            if (sg[r] == 0) continue; /* singular block: contribution dropped */
            double w = coef[r] * psi[r];
            net_forward(n, S[2 * r], S[2 * r + 1], x, h1, h2, phi);
            occ_list(S[2 * r], norb, oa);
            occ_list(S[2 * r + 1], norb, ob);
            memset(dphi, 0, sizeof(double) * nout);
            double la;
            gather_block(phi, nel, oa, n->na, 0, A);
            lu_factor(A, n->na, perm, &la);
            lu_inverse(A, perm, n->na, inv);
            for (int j = 0; j < n->na; ++j)
                for (int k = 0; k < n->na; ++k)
                    dphi[(size_t)oa[j] * nel + k] += w * inv[k * n->na + j];
            gather_block(phi, nel, ob, n->nb, n->na, A);
            lu_factor(A, n->nb, perm, &la);
            lu_inverse(A, perm, n->nb, inv);
            for (int j = 0; j < n->nb; ++j)
                for (int k = 0; k < n->nb; ++k)
                    dphi[(size_t)ob[j] * nel + n->na + k] += w * inv[k * n->nb + j];
            /* output layer */
            for (int i = 0; i < n->H2; ++i) dh2[i] = 0.0;
            for (int o = 0; o < nout; ++o) {
                double d = dphi[o];
                if (d == 0.0) continue;
                gb3[o] += d;
                for (int k = 0; k < n->H2; ++k) {
                    gW3[(size_t)o * n->H2 + k] += d * h2[k];
                    dh2[k] += wq(n, n->W3[(size_t)o * n->H2 + k]) * d;
                }
            }
            /* hidden layer 2: tanh' = 1 - h^2 */
            for (int i = 0; i < n->H1; ++i) dh1[i] = 0.0;
            for (int i = 0; i < n->H2; ++i) {
                double dz = dh2[i] * (1.0 - h2[i] * h2[i]);
                gb2[i] += dz;
                for (int k = 0; k < n->H1; ++k) {
                    gW2[(size_t)i * n->H1 + k] += dz * h1[k];
                    dh1[k] += wq(n, n->W2[(size_t)i * n->H1 + k]) * dz;
                }
            }
            /* hidden layer 1 */
            for (int i = 0; i < n->H1; ++i) {
                double dz = dh1[i] * (1.0 - h1[i] * h1[i]);
                gb1[i] += dz;
                for (int k = 0; k < nin; ++k) gW1[(size_t)i * nin + k] += dz * x[k];
            }
        }
        free(x);
        free(h1);
        free(h2);
        free(phi);
        free(dphi);
        free(dh2);
        free(dh1);
    }
    for (int64_t p = 0; p < np; ++p) {
        double s = 0.0;
        for (int t = 0; t < nthr; ++t) s += acc[(size_t)np * t + p];
        grad[p] = s;
    }
    free(acc);
    return ORC_OK;
}

int orc_energy_grad(const orc_net* n, const uint64_t* S, int64_t nS, const int64_t* row_ptr,
                    const int32_t* col, const double* val, double* out, double* grad,
                    double* psi_out, double* v_out) {
    if (nS <= 0) return ORC_ERR_ARG;
    double* logabs = (double*)malloc(sizeof(double) * nS);
    int8_t* sg = (int8_t*)malloc(nS);
    double* psi = (double*)malloc(sizeof(double) * nS);
    double* v = (double*)malloc(sizeof(double) * nS);
    if (!logabs || !sg || !psi || !v) return ORC_ERR_OOM;
    int status = orc_amplitudes(n, S, nS, logabs, sg);
    double M = -INFINITY;
    for (int64_t r = 0; r < nS; ++r)
        if (sg[r] != 0 && logabs[r] > M) M = logabs[r];
    for (int64_t r = 0; r < nS; ++r) psi[r] = sg[r] == 0 ? 0.0 : sg[r] * exp(logabs[r] - M);
    double ev[3];
    orc_energy_from_psi(row_ptr, col, val, psi, nS, ev, v);
    out[0] = ev[0];
    out[1] = ev[1];
    out[2] = ev[2];
    out[3] = M;
    double E = ev[0], D = ev[2];
    if (grad) {
        double* coef = (double*)malloc(sizeof(double) * nS);
        if (!coef) return ORC_ERR_OOM;
        for (int64_t r = 0; r < nS; ++r) coef[r] = (2.0 / D) * (v[r] - E * psi[r]);
        int st = grad_core(n, S, nS, sg, psi, coef, grad);
        free(coef);
        if (st != ORC_OK) return st;
    }
    if (psi_out) memcpy(psi_out, psi, sizeof(double) * nS);
    if (v_out) memcpy(v_out, v, sizeof(double) * nS);
    free(logabs);
    free(sg);
    free(psi);
    free(v);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Asymmetric mode (Sec. 2.4.1, Eqs. asymmetric_energy, asymmetric_gradient) on T = V + P with
 * the proxy CSR over T (its V rows hold every connection inside T; its P rows the connections to
 * V after their diagonal):
 *   E_asym = N / D,  N = sum_{x in V} psi_x (H_VT psi_T)_x,  D = sum_{x in V} psi_x^2
 *     (= sum_V p_V(x) E_loc(x) with E_loc(x) = (H_VT psi_T)_x / psi_x).
 * Gradient, as sum over z in T of c_z d psi_z / d theta:
 *   exact = 0:  the log-derivative estimator of Eq. (asymmetric_gradient):
 *               c_z = 2 ((H_VT psi)_z - E psi_z) / D for z in V, 0 for z in P;
 *   exact = 1:  the derivative of E_asym itself (dependence through psi_P included):
 *               c_z = ((H_VT psi)_z + (H_VV psi_V)_z - 2 E psi_z) / D  for z in V,
 *               c_z = (H_PV psi_V)_z / D                              for z in P.
 * psi is scaled by exp(-max over T of log|psi|). out = [E, N, D, max log|psi|].
 * ---------------------------------------------------------------------------------------- */
int orc_asym_energy_grad(const orc_net* n, const uint64_t* T, int64_t nT, int64_t nV,
                         const int64_t* row_ptr, const int32_t* col, const double* val,
                         int exact, double* out, double* grad) {
    if (nV <= 0 || nT < nV) return ORC_ERR_ARG;
    double* logabs = (double*)malloc(sizeof(double) * nT);
    int8_t* sg = (int8_t*)malloc(nT);
    double* psi = (double*)malloc(sizeof(double) * nT);
    double* c = (double*)malloc(sizeof(double) * nT);
    if (!logabs || !sg || !psi || !c) return ORC_ERR_OOM;
    int status = orc_amplitudes(n, T, nT, logabs, sg);
    double M = -INFINITY;
    for (int64_t r = 0; r < nT; ++r)
        if (sg[r] != 0 && logabs[r] > M) M = logabs[r];
    for (int64_t r = 0; r < nT; ++r) psi[r] = sg[r] == 0 ? 0.0 : sg[r] * exp(logabs[r] - M);
    /* row sums: all of row x (H_VT psi), its V columns (H_VV psi_V), P rows without diagonal */
    double* v_all = (double*)malloc(sizeof(double) * nT);
    double* v_in = (double*)malloc(sizeof(double) * nT);
    if (!v_all || !v_in) return ORC_ERR_OOM;
    for (int64_t r = 0; r < nT; ++r) {
        double sa = 0.0, si = 0.0;
        for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            double t = val[k] * psi[col[k]];
            if (r >= nV && k == row_ptr[r]) continue; /* the diagonal of a P row */
            sa += t;
            if (col[k] < nV) si += t;
        }
        v_all[r] = sa;
        v_in[r] = si;
    }
    ksum Nk = {0, 0}, Dk = {0, 0};
    for (int64_t r = 0; r < nV; ++r) {
        kadd(&Nk, psi[r] * v_all[r]);
        kadd(&Dk, psi[r] * psi[r]);
    }
    double N = kval(&Nk), D = kval(&Dk), E = N / D;
    out[0] = E;
    out[1] = N;
    out[2] = D;
    out[3] = M;
    if (grad) {
        for (int64_t r = 0; r < nT; ++r) {
            if (r < nV)
                c[r] = exact ? (v_all[r] + v_in[r] - 2.0 * E * psi[r]) / D
                             : 2.0 * (v_all[r] - E * psi[r]) / D;
            else
                c[r] = exact ? v_all[r] / D : 0.0;
        }
        int st = grad_core(n, T, nT, sg, psi, c, grad);
        if (st != ORC_OK) return st;
    }
    free(logabs);
    free(sg);
    free(psi);
    free(c);
    free(v_all);
    free(v_in);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Bucket function for hash-partitioned PT2: SplitMix64's output finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), applied as
 * h = mix(mix(a) ^ b), and bucket(a, b) = floor(floor(h / 2^32) * B / 2^32) for B < 2^32 (the
 * high 32 bits of h scaled to [0, B)). Part of the interface, restated on each side.
 * ---------------------------------------------------------------------------------------- */
static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
uint64_t orc_bucket(uint64_t a, uint64_t b, uint64_t nbuckets) {
    const uint64_t h = mix64(mix64(a) ^ b);
    return ((h >> 32) * nbuckets) >> 32;
}

/* ------------------------------------------------------------------------------------------
 * Epstein-Nesbet PT2 (Eq. pt2_correction), with Psi_V normalised by D = psi^T psi:
 *   external: sum over x' in C\S of c(x')^2 / (D (E - H_x'x')),  c(x') = sum_{y in S} H_x'y psi_y
 *   internal: sum over x in S of r_x^2 / (D (E - H_xx)),          r = H_SS psi - E psi
 * c(x') is accumulated by emitting (x', H_x'y psi_y) for every excitation of every y in S
 * (y ascending), sorting by (key, emission number) and summing each run in order. The
 * external sum runs in ascending key order, the internal in S order, both compensated.
 * bucket >= 0 restricts both terms to configurations x with bucket(x) == bucket.
 * out = [dE_ext, dE_int, n_unique_external, D, number of emitted pairs].
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    uint64_t a, b;
    double v;
    int64_t seq;
} emit_t;

static int emit_cmp(const void* p, const void* q) {
    const emit_t* x = (const emit_t*)p;
    const emit_t* y = (const emit_t*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    return 0;
}

int orc_pt2_eps(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                const double* psi, double E, double eps, int64_t nbuckets, int64_t bucket,
                double* out);
int orc_pt2(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
            const double* psi, double E, int64_t nbuckets, int64_t bucket, double* out) {
    return orc_pt2_eps(norb, h, eri, S, nS, psi, E, 0.0, nbuckets, bucket, out);
}

/* emission test of the screened form: targets inside S always (the internal term is exact);
 * targets outside S when |H_x'y| |psi_y| >= eps (every one when eps = 0) */
static int pt2_keep(const uint64_t* S, int64_t nS, uint64_t xa, uint64_t xb, double hv,
                    double py, double eps) {
    if (eps == 0.0) return 1;
    if (fabs(hv) * fabs(py) >= eps) return 1;
    return find_in_S(S, nS, xa, xb) >= 0;
}

/* The same correction with the external sum screened as in Sec. 3.3 (Eq. hb_screen applied to
 * each contribution): c(x') keeps only the terms H_x'y psi_y with |H_x'y psi_y| >= eps, and the
 * external sum runs over the x' outside S that receive at least one such term (the screened
 * perturbative set P). The internal term stays exact. eps = 0 is orc_pt2. */
static int pt2_core(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                    const double* psi, double E, double eps, int64_t nbuckets, int64_t bucket,
                    double* out, int64_t cap, uint64_t* keys_out, double* c_out);

int orc_pt2_eps(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                const double* psi, double E, double eps, int64_t nbuckets, int64_t bucket,
                double* out) {
    return pt2_core(norb, h, eri, S, nS, psi, E, eps, nbuckets, bucket, out, 0, NULL, NULL);
}

/* The unique external set of the same reduction: for every x' in C\S (of bucket `bucket`, or
 * all when bucket < 0), in ascending key order, the configuration (keys_out[2k], keys_out[2k+1])
 * and c(x') = sum_{y in S} H_x'y psi_y (c_out[k]), for k < min(n_unique, cap). out as in
 * orc_pt2_eps; returns ORC_OK. */
int orc_pt2_unique(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                   const double* psi, double E, int64_t nbuckets, int64_t bucket, double* out,
                   int64_t cap, uint64_t* keys_out, double* c_out) {
    return pt2_core(norb, h, eri, S, nS, psi, E, 0.0, nbuckets, bucket, out, cap, keys_out,
                    c_out);
}

/* the same set for the screened sum (contributions with |H_x'y| |psi_y| >= eps kept, Sec. 3.3):
 * x' reached by at least one kept contribution, c(x') the sum of those */
int orc_pt2_unique_eps(int norb, const double* h, const double* eri, const uint64_t* S,
                       int64_t nS, const double* psi, double E, double eps, int64_t nbuckets,
                       int64_t bucket, double* out, int64_t cap, uint64_t* keys_out,
                       double* c_out) {
    return pt2_core(norb, h, eri, S, nS, psi, E, eps, nbuckets, bucket, out, cap, keys_out,
                    c_out);
}

static int pt2_core(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                    const double* psi, double E, double eps, int64_t nbuckets, int64_t bucket,
                    double* out, int64_t cap, uint64_t* keys_out, double* c_out) {
    if (nS <= 0 || nbuckets < 1 || !(eps >= 0.0)) return ORC_ERR_ARG;
    int na = popc(S[0]), nb = popc(S[1]);
    int64_t nexc = orc_n_excitations(norb, na, nb);
    ksum Dk = {0, 0};
    for (int64_t r = 0; r < nS; ++r) kadd(&Dk, psi[r] * psi[r]);
    double D = kval(&Dk);
    /* count emissions per parent, then emit in parent order */
    int64_t* cnt = (int64_t*)calloc(nS + 1, sizeof(int64_t));
    if (!cnt) return ORC_ERR_OOM;
#pragma omp parallel
    {
        uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * 2 * nexc);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nS; ++r) {
            int64_t n = orc_excitations(norb, S[2 * r], S[2 * r + 1], buf), c = 0;
            for (int64_t k = 0; k < n; ++k) {
                uint64_t xa = buf[2 * k], xb = buf[2 * k + 1];
                if (bucket >= 0 && (int64_t)orc_bucket(xa, xb, nbuckets) != bucket) continue;
                double hv = eps == 0.0 ? 0.0
                                       : orc_element(norb, h, eri, S[2 * r], S[2 * r + 1], xa, xb,
                                                     NULL);
                if (pt2_keep(S, nS, xa, xb, hv, psi[r], eps)) ++c;
            }
            cnt[r + 1] = c;
        }
        free(buf);
    }
    for (int64_t r = 0; r < nS; ++r) cnt[r + 1] += cnt[r];
    int64_t total = cnt[nS];
    emit_t* em = (emit_t*)malloc(sizeof(emit_t) * (total > 0 ? total : 1));
    if (!em) {
        free(cnt);
        return ORC_ERR_OOM;
    }
#pragma omp parallel
    {
        uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * 2 * nexc);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nS; ++r) {
            uint64_t a = S[2 * r], b = S[2 * r + 1];
            int64_t n = orc_excitations(norb, a, b, buf), pos = cnt[r];
            for (int64_t k = 0; k < n; ++k) {
                uint64_t xa = buf[2 * k], xb = buf[2 * k + 1];
                if (bucket >= 0 && (int64_t)orc_bucket(xa, xb, nbuckets) != bucket) continue;
                double hv = orc_element(norb, h, eri, a, b, xa, xb, NULL);
                if (!pt2_keep(S, nS, xa, xb, hv, psi[r], eps)) continue;
                em[pos].a = xa;
                em[pos].b = xb;
                em[pos].v = hv * psi[r];
                em[pos].seq = pos;
                ++pos;
            }
        }
        free(buf);
    }
    qsort(em, total, sizeof(emit_t), emit_cmp);
    double* cS = (double*)calloc(nS, sizeof(double));
    ksum ext = {0, 0};
    int64_t nuniq = 0;
    for (int64_t k = 0; k < total;) {
        int64_t e = k;
        double c = 0.0;
        while (e < total && em[e].a == em[k].a && em[e].b == em[k].b) {
            c += em[e].v;
            ++e;
        }
        int64_t s = find_in_S(S, nS, em[k].a, em[k].b);
        if (s >= 0) {
            cS[s] = c;
        } else {
            double hxx = orc_diag(norb, h, eri, em[k].a, em[k].b);
            kadd(&ext, (c * c) / (D * (E - hxx)));
            if (nuniq < cap) {
                keys_out[2 * nuniq] = em[k].a;
                keys_out[2 * nuniq + 1] = em[k].b;
                c_out[nuniq] = c;
            }
            ++nuniq;
        }
        k = e;
    }
    ksum in = {0, 0};
    for (int64_t r = 0; r < nS; ++r) {
        uint64_t a = S[2 * r], b = S[2 * r + 1];
        if (bucket >= 0 && (int64_t)orc_bucket(a, b, nbuckets) != bucket) continue;
        double hxx = orc_diag(norb, h, eri, a, b);
        double vx = hxx * psi[r] + cS[r];
        double rr = vx - E * psi[r];
        kadd(&in, (rr * rr) / (D * (E - hxx)));
    }
    out[0] = kval(&ext);
    out[1] = kval(&in);
    out[2] = (double)nuniq;
    out[3] = D;
    out[4] = (double)total;
    free(cS);
    free(em);
    free(cnt);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Proxy Hamiltonian of Eq. (proxy_hamiltonian) (Sec. 2.4.1, Proxy mode) on T = V + P as a CSR
 * over T, with T[0..nV) = V and T[nV..nT) = P, each sorted by key:
 *   (H~)_xy = H_xy when x or y is in V;  H_xx on the diagonal;  0 for x != y both in P.
 * Row x in V: [diagonal, then every excitation of x found in T, canonical order]; row x in P:
 * [diagonal, then every excitation of x found in V, ascending V index]. Column = index in T.
 * With this matrix E_proxy (Eq. proxy_energy) and its gradient (Eq. proxy_gradient) are the
 * Rayleigh quotient and gradient of orc_energy_grad over T. Two passes like orc_hss.
 * ---------------------------------------------------------------------------------------- */
static int64_t find_in_T(const uint64_t* T, int64_t nV, int64_t nT, uint64_t a, uint64_t b) {
    int64_t v = find_in_S(T, nV, a, b);
    if (v >= 0) return v;
    int64_t q = find_in_S(T + 2 * nV, nT - nV, a, b);
    return q >= 0 ? nV + q : -1;
}

typedef struct {
    int64_t c;
    double v;
} colval_t;

static int colval_cmp(const void* p, const void* q) {
    int64_t a = ((const colval_t*)p)->c, b = ((const colval_t*)q)->c;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_proxy_csr(int norb, const double* h, const double* eri, const uint64_t* T, int64_t nV,
                  int64_t nT, int fill, int64_t* row_ptr, int32_t* col, double* val) {
    if (norb < 1 || norb > 64 || nV < 0 || nT < nV) return ORC_ERR_ARG;
    if (nT == 0) {
        row_ptr[0] = 0;
        return ORC_OK;
    }
    int na = popc(T[0]), nb = popc(T[1]);
    int64_t nexc = orc_n_excitations(norb, na, nb);
    int err = 0;
#pragma omp parallel
    {
        uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)(nexc > 0 ? nexc : 1));
        colval_t* cv = (colval_t*)malloc(sizeof(colval_t) * (size_t)(nexc > 0 ? nexc : 1));
        if (!buf || !cv) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nT; ++r) {
            if (!buf || !cv) continue;
            uint64_t a = T[2 * r], b = T[2 * r + 1];
            int64_t n = orc_excitations(norb, a, b, buf), m = 0;
            for (int64_t k = 0; k < n; ++k) {
                int64_t c = r < nV ? find_in_T(T, nV, nT, buf[2 * k], buf[2 * k + 1])
                                   : find_in_S(T, nV, buf[2 * k], buf[2 * k + 1]);
                if (c < 0) continue;
                cv[m].c = c;
                cv[m].v = fill ? orc_element(norb, h, eri, a, b, buf[2 * k], buf[2 * k + 1], NULL)
                               : 0.0;
                ++m;
            }
            if (!fill) {
                row_ptr[r + 1] = m + 1;
                continue;
            }
            if (r >= nV) qsort(cv, m, sizeof(colval_t), colval_cmp);
            int64_t pos = row_ptr[r];
            col[pos] = (int32_t)r;
            val[pos] = orc_diag(norb, h, eri, a, b);
            for (int64_t k = 0; k < m; ++k) {
                col[pos + 1 + k] = (int32_t)cv[k].c;
                val[pos + 1 + k] = cv[k].v;
            }
        }
        free(buf);
        free(cv);
    }
    if (err) return ORC_ERR_OOM;
    if (!fill) {
        row_ptr[0] = 0;
        for (int64_t r = 0; r < nT; ++r) row_ptr[r + 1] += row_ptr[r];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * Heat-bath screened perturbative set, Eq. (hb_screen) of Sec. 3.3:
 *   P = { x' not in S : max over x in S of |H_x'x psi(x)| >= eps }.
 * Written as that definition: every excitation x' of every x in S gets its Slater-Condon
 * element; the pair is kept when |H_x'x| * |psi_x| >= eps (one FP64 product) and x' is not in
 * S; the kept pairs are sorted by key and each run reduced to its maximum. (The sorted-table
 * early exit of Sec. 3.3 is an acceleration of the same test and is not used here.)
 * Writes keys[n][2] (ascending) and mx[n] = max_x |H_x'x| |psi_x| when cap >= n.
 * Returns n, or a negative status.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    uint64_t a, b;
    double m;
} hb_t;

static int hb_cmp(const void* p, const void* q) {
    const hb_t* x = (const hb_t*)p;
    const hb_t* y = (const hb_t*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

int64_t orc_hb_select_rows(int norb, const double* h, const double* eri, const uint64_t* S,
                           int64_t nS, int64_t r0, int64_t r1, const double* psi, double eps,
                           int64_t cap, uint64_t* keys, double* mx);
int64_t orc_hb_select(int norb, const double* h, const double* eri, const uint64_t* S, int64_t nS,
                      const double* psi, double eps, int64_t cap, uint64_t* keys, double* mx) {
    return orc_hb_select_rows(norb, h, eri, S, nS, 0, nS, psi, eps, cap, keys, mx);
}

/* The same with the maximum taken over the parents x = S[r0..r1-1] only (membership is still
 * tested against all of S): a subset of P whose couplings are lower bounds of P's. */
int64_t orc_hb_select_rows(int norb, const double* h, const double* eri, const uint64_t* S,
                           int64_t nS, int64_t r0, int64_t r1, const double* psi, double eps,
                           int64_t cap, uint64_t* keys, double* mx) {
    if (nS <= 0 || !(eps >= 0.0) || r0 < 0 || r1 > nS || r0 > r1) return ORC_ERR_ARG;
    int na = popc(S[0]), nb = popc(S[1]);
    int64_t nexc = orc_n_excitations(norb, na, nb);
    int64_t* cnt = (int64_t*)calloc(nS + 1, sizeof(int64_t));
    if (!cnt) return ORC_ERR_OOM;
    /* pass 1 counts the kept pairs of each x, pass 2 writes them at the prefix offsets */
    hb_t* kept = NULL;
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel
        {
            uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * 2 * nexc);
#pragma omp for schedule(dynamic, 16)
            for (int64_t r = r0; r < r1; ++r) {
                uint64_t a = S[2 * r], b = S[2 * r + 1];
                int64_t n = orc_excitations(norb, a, b, buf), c = 0;
                for (int64_t k = 0; k < n; ++k) {
                    uint64_t xa = buf[2 * k], xb = buf[2 * k + 1];
                    double hv = orc_element(norb, h, eri, a, b, xa, xb, NULL);
                    double m = fabs(hv) * fabs(psi[r]);
                    if (!(m >= eps) || find_in_S(S, nS, xa, xb) >= 0) continue;
                    if (pass == 1) {
                        kept[cnt[r] + c].a = xa;
                        kept[cnt[r] + c].b = xb;
                        kept[cnt[r] + c].m = m;
                    }
                    ++c;
                }
                if (pass == 0) cnt[r + 1] = c;
            }
            free(buf);
        }
        if (pass == 0) {
            for (int64_t r = 0; r < nS; ++r) cnt[r + 1] += cnt[r];  /* rows outside stay 0 */
            kept = (hb_t*)malloc(sizeof(hb_t) * (cnt[nS] > 0 ? cnt[nS] : 1));
            if (!kept) {
                free(cnt);
                return ORC_ERR_OOM;
            }
        }
    }
    int64_t total = cnt[nS];
    qsort(kept, total, sizeof(hb_t), hb_cmp);
    int64_t n = 0;
    for (int64_t k = 0; k < total;) {
        int64_t e = k;
        double m = kept[k].m;
        while (e < total && kept[e].a == kept[k].a && kept[e].b == kept[k].b) {
            if (kept[e].m > m) m = kept[e].m;
            ++e;
        }
        if (keys && mx && n < cap) {
            keys[2 * n] = kept[k].a;
            keys[2 * n + 1] = kept[k].b;
            mx[n] = m;
        }
        ++n;
        k = e;
    }
    free(kept);
    free(cnt);
    return n;
}

/* ------------------------------------------------------------------------------------------
 * Subspace selection of the outer loop (Sec. 2.4.2; Algorithm 1 step 3, Selector(T, K,
 * key = |psi|)). Input: the amplitudes on T as log|psi| (-inf for psi = 0). The configurations
 * are ranked by log|psi| descending, ties by ascending key, and a prefix of the ranking is kept.
 * With w_x = exp(2 (log|psi_x| - max log|psi|)) (psi^2 up to one common factor) and
 * D = sum over T of w (compensated, in T order):
 *   mode 0  Top-K:              the first min(K, n);
 *   mode 1  cumulative mass:    the shortest prefix whose sum of w (added in rank order)
 *                               reaches gamma * D; all of T if rounding keeps it below;
 *   mode 2  absolute threshold: every x with p(x) = w_x / D > eps (a prefix of the ranking).
 * Writes the positions in T of the kept configurations, ascending by key, and returns their
 * number (or a negative status).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    uint64_t a, b;
    double m;
    int64_t pos;
} rank_t;

static int rank_cmp(const void* p, const void* q) {
    const rank_t* x = (const rank_t*)p;
    const rank_t* y = (const rank_t*)q;
    if (x->m != y->m) return x->m > y->m ? -1 : 1;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

static int key_cmp(const void* p, const void* q) {
    const rank_t* x = (const rank_t*)p;
    const rank_t* y = (const rank_t*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

int64_t orc_select(const uint64_t* T, const double* logabs, int64_t n, int mode, int64_t K,
                   double param, int64_t* out_pos) {
    if (n <= 0 || mode < 0 || mode > 2) return ORC_ERR_ARG;
    rank_t* r = (rank_t*)malloc(sizeof(rank_t) * n);
    if (!r) return ORC_ERR_OOM;
    double lmax = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        r[i].a = T[2 * i];
        r[i].b = T[2 * i + 1];
        r[i].m = logabs[i];
        r[i].pos = i;
        if (logabs[i] > lmax) lmax = logabs[i];
    }
    ksum Dk = {0, 0};
    for (int64_t i = 0; i < n; ++i) kadd(&Dk, exp(2.0 * (logabs[i] - lmax)));
    double D = kval(&Dk);
    qsort(r, n, sizeof(rank_t), rank_cmp);
    int64_t c = 0;
    if (mode == 0) {
        c = K < n ? (K > 0 ? K : 0) : n;
    } else if (mode == 1) {
        double target = param * D, acc = 0.0;
        c = n;
        for (int64_t i = 0; i < n; ++i) {
            acc = acc + exp(2.0 * (r[i].m - lmax));
            if (acc >= target) {
                c = i + 1;
                break;
            }
        }
    } else {
        while (c < n && exp(2.0 * (r[c].m - lmax)) / D > param) ++c;
    }
    qsort(r, c, sizeof(rank_t), key_cmp);
    for (int64_t i = 0; i < c; ++i) out_pos[i] = r[i].pos;
    free(r);
    return c;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
