/*
 * nqs.h -- C ABI of the B300 (sm_103a) library for the data-parallel hot path of the
 * deterministic neural-network-quantum-state method of arXiv 2601.21310:
 *   (1) Slater-Condon generation of all single and double excitations of the configurations
 *       of a selected set S, with fermionic signs and FP64 matrix elements, and the projected
 *       Hamiltonian H_SS in CSR (Sec. 3.1 "Discrete Combinatorial Kernel"; Eq. connected_set);
 *   (2) the neural-backflow amplitude psi(x) = det Phi(x)[occ_a, 0:na] * det Phi(x)[occ_b,
 *       na:na+nb] with Phi(x) = Phi0 + MLP(x) (Eqs. effective_orbital_matrix,
 *       occupied_submatrix, backflow_amplitude);
 *   (3) the subspace variational energy E_S and its parameter gradient (Eqs.
 *       variational_energy, variational_gradient);
 *   (4) the post-hoc Epstein-Nesbet PT2 correction over C\S (Eq. pt2_correction).
 *
 * Conventions shared by every entry point
 *   - A configuration ("det") is two uint64 words {a, b}: bit p of a (b) set means alpha (beta)
 *     spatial orbital p is occupied. Arrays of dets are [n][2] uint64, 16-byte aligned.
 *   - Key order is (a, b) lexicographic with a in the high word. S must be sorted ascending
 *     and unique, and every det must hold nalpha alpha and nbeta beta electrons.
 *   - Spin-orbital order is alpha 0..norb-1 then beta 0..norb-1, and |x> is the product of
 *     creation operators of the occupied spin-orbitals in ascending order acting on |0>. Under
 *     this order the single-excitation sign is (-1)^(occupied orbitals of that spin strictly
 *     between the two indices).
 *   - ERIs are real, in chemists' notation (pq|rs), with eightfold symmetry, stored row-major
 *     as eri[((p*norb+q)*norb+r)*norb+s].
 *   - Canonical excitation order of one det: alpha singles (i asc, a asc), beta singles,
 *     alpha-alpha doubles (hole pairs i<j lexicographic, then particle pairs a<b
 *     lexicographic), beta-beta doubles, alpha-beta doubles (i_a, a_a, j_b, b_b, b fastest).
 *   - Pointers marked "device" are CUDA device pointers of the current device; "host" are
 *     ordinary host pointers. Unless stated, the caller owns every buffer it passes.
 *   - All work is ordered on the given stream (NULL = legacy default stream). Calls that
 *     return host scalars synchronise that stream before returning.
 *   - Every function returns NQS_OK (0), a positive warning, or a negative error code; no
 *     C++ exception crosses this boundary. On error, outputs are unspecified.
 *   - Handles are not thread safe: use one problem handle from one host thread at a time.
 */
#ifndef NQS_H
#define NQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* nqs_stream_t; /* the same object as cudaStream_t */

/* ---- status codes ------------------------------------------------------------------------ */
#define NQS_OK 0
#define NQS_WARN_SINGULAR 1        /* an occupied block had an exactly zero pivot: psi = 0 */
#define NQS_ERR_ARG (-1)           /* invalid argument (null pointer, size, option) */
#define NQS_ERR_UNSORTED (-2)      /* S is not sorted ascending or has duplicates */
#define NQS_ERR_POPCOUNT (-3)      /* a det has the wrong number of alpha/beta electrons */
#define NQS_ERR_NORB (-4)          /* norb outside 1..64, or key wider than supported */
#define NQS_ERR_OOM (-5)           /* device allocation failed */
#define NQS_ERR_CUDA (-6)          /* a CUDA runtime call or a kernel launch failed */
#define NQS_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up */
#define NQS_ERR_UNSUPPORTED (-8)   /* valid request outside what the library implements */

/* ---- precision forms -------------------------------------------------------------------- */
#define NQS_FP64 0   /* plain form: FP64 parameters, FP64 GEMMs, FP64 LU */
#define NQS_MIXED 1  /* BF16 weights and activations on tensor cores with FP32 accumulation,
                        FP32 biases/Phi0, FP32 LU with FP64 log|det|; FP64 for everything
                        Hamiltonian-side (elements, SpMV, reductions, PT2) */

typedef struct nqs_problem nqs_problem; /* opaque: device copies of the integrals */
typedef struct nqs_net nqs_net;         /* opaque: refers to caller-owned device parameters */

/* Options. Zero-initialise and set what you need; nqs_opts_default() fills the defaults. */
typedef struct {
    int precision;      /* NQS_FP64 or NQS_MIXED (must match the net's dtype) */
    int buckets;        /* PT2 hash buckets, >= 1 (more buckets = less scratch memory) */
    int64_t chunk;      /* PT2 cap on emitted (key, value) pairs per sorted bucket, and on the
                           slots of a hashed pass's table; 0 = automatic (from free memory) */
    int validate;       /* 1: check that S is sorted, unique and has the right popcounts */
    int internal_pt2;   /* 1: also compute the internal (x in S) PT2 term */
    double eps_pt2;     /* PT2 screening (Sec. 3.3 criterion per contribution): 0 = the full
                           connected space; > 0 keeps only the external contributions
                           |H_x'y psi_y| >= eps_pt2 (psi as passed to nqs_pt2), so the external
                           sum runs over the screened perturbative set; the internal term stays
                           exact */
    int batch_log2;     /* micro-batch of the amplitude and energy paths, 2^batch_log2
                           configurations (0 = 2^20). Larger sets are evaluated batch by batch,
                           and their gradient recomputes each batch's activations (Sec. 3.2:
                           gradients accumulated over fixed-size micro-batches), so activation
                           memory is bounded by the batch. */
    int reserved[5];
} nqs_opts;

/* Library-owned CSR of H_SS (device memory). Row r holds, in order: the diagonal element
 * (column r), then every excitation of S[r] that lies in S, in canonical excitation order.
 * val[k] = <S[col[k]]|H|S[r]> (H_SS is symmetric, bit for bit under this library's summation
 * order). Free with nqs_csr_free or nqs_csr_free_async. */
typedef struct {
    int64_t* row_ptr; /* device [n_rows + 1] */
    int32_t* col;     /* device [nnz] */
    double* val;      /* device [nnz] */
    int64_t nnz;
    int64_t n_rows;
} nqs_csr;

void nqs_opts_default(nqs_opts* opts);
const char* nqs_status_string(int status);
const char* nqs_version(void);
/* message of the last failed CUDA call on this host thread ("" if none) */
const char* nqs_last_error(void);

/* Build the problem: copies h (host, norb*norb FP64, symmetric) and eri (host, norb^4 FP64,
 * chemists' notation) to the current device, with derived tables (Coulomb J_pq = (pp|qq),
 * exchange K_pq = (pq|qp)). ecore is added to nothing: energies are electronic. Requires
 * 1 <= norb <= 64 and 0 < nalpha, nbeta < norb. Synchronous. Errors: NQS_ERR_ARG,
 * NQS_ERR_NORB, NQS_ERR_OOM, NQS_ERR_CUDA. Sec. 3.3 (Hamiltonian integrals as input),
 * Algorithm 1 input. */
int nqs_problem_create(int norb, int nalpha, int nbeta, const double* h, const double* eri,
                       double ecore, nqs_problem** out);
int nqs_problem_destroy(nqs_problem* problem);

/* Describe the backflow network of Sec. 2.2 / Sec. 3.3: input x in {0,1}^(2 norb) (alpha bits
 * then beta bits), z1 = W1 x + b1, h1 = tanh z1, z2 = W2 h1 + b2, h2 = tanh z2,
 * out = W3 h2 + b3, Phi = Phi0 + reshape(out, [norb][na+nb]) row-major.
 * params: 7 device pointers {W1 [H1][2 norb], b1 [H1], W2 [H2][H1], b2 [H2],
 * W3 [norb(na+nb)][H2], b3 [norb(na+nb)], Phi0 [norb][na+nb]}, all row-major, owned by the
 * caller and read at every call (so optimiser updates in place are seen).
 * dtype NQS_FP64: all FP64. dtype NQS_MIXED: W1, W2, W3 bfloat16; b1, b2, b3, Phi0 float.
 * Phi0 is fixed (not differentiated). Errors: NQS_ERR_ARG, NQS_ERR_OOM. */
int nqs_net_create(nqs_problem* problem, int H1, int H2, int dtype, const void* const* params,
                   nqs_net** out);
int nqs_net_destroy(nqs_net* net);
/* number of trainable parameters = H1*2norb + H1 + H2*H1 + H2 + nout*H2 + nout */
int64_t nqs_net_num_params(const nqs_net* net);

/* H_xx for n dets (Slater-Condon, zero excitations; the denominators of Eq. pt2_correction).
 * dets: device [n][2]; out: device [n] FP64. Stream-ordered, no sync. */
int nqs_diag(nqs_problem* problem, const uint64_t* dets, int64_t n, double* out,
             nqs_stream_t stream);

/* Resolve every single and double excitation of every det of S (Eq. connected_set) as a member
 * of S or not, and build H_SS in CSR (Sec. 3.1: the combinatorial kernel exports H_VV as CSR;
 * Algorithm 1 step 1). Membership comes from a hash table of S and, for whole blocks of
 * excitations at once, from indices of S by alpha string and by beta string (a det's beta
 * excitations are the members of its own alpha run that differ in 2 or 4 beta bits, and so
 * on); the result is the same as looking up each excitation. Rows: the diagonal, then the hits
 * in canonical excitation order. dets: device [nS][2], sorted and unique. On success *out holds
 * a library-owned CSR and *n_enumerated (host, may be NULL) the number of (det, excitation)
 * pairs resolved (nS times the excitations per det). Device scratch from the problem's pool:
 * the hash table (22 B per slot, 16 to 32 slots per det up to 2^22 dets, fewer above), the two
 * indices (80 to 152 B per det) and the hit ballots (4 B per 32 excitations per det).
 * Synchronises the stream (nnz must be known to allocate). Errors: NQS_ERR_ARG,
 * NQS_ERR_UNSORTED / NQS_ERR_POPCOUNT (with validate), NQS_ERR_OOM, NQS_ERR_CUDA. */
int nqs_connections(nqs_problem* problem, const uint64_t* dets, int64_t nS, const nqs_opts* opts,
                    nqs_csr* out, int64_t* n_enumerated, nqs_stream_t stream);
/* Release a library-owned CSR (from nqs_connections or nqs_proxy_hamiltonian; its arrays come
 * from the problem's stream-ordered pool, which outlives the problem handle while they exist).
 * nqs_csr_free waits for the whole device first. nqs_csr_free_async releases the arrays in the
 * order of `stream`: work already queued on that stream may still read them, and work on other
 * streams must be ordered before it by the caller. Both zero *csr. Errors: NQS_ERR_ARG,
 * NQS_ERR_CUDA. */
int nqs_csr_free(nqs_csr* csr);
int nqs_csr_free_async(nqs_csr* csr, nqs_stream_t stream);

/* Proxy-mode Hamiltonian, Eq. (proxy_hamiltonian) of Sec. 2.4.1, on the target set T = V + P:
 * (H~)_xy = H_xy when x or y lies in V, H_xx on the diagonal, 0 between distinct members of P.
 * T: device [nT][2] with T[0..nV) = V and T[nV..nT) = P, each sorted by key and disjoint
 * (both checked with opts->validate). On success *out holds a library-owned CSR over T (free with
 * nqs_csr_free): row x of V = [diagonal, then every excitation of x found in T, canonical order];
 * row x of P = [diagonal, then the members of V connected to x, ascending]; columns are positions
 * in T; symmetric bit for bit. nqs_energy_grad over T with this matrix gives E_proxy
 * (Eq. proxy_energy) and its gradient (Eq. proxy_gradient). Synchronises the stream. Errors:
 * NQS_ERR_ARG, NQS_ERR_UNSORTED / NQS_ERR_POPCOUNT (with validate), NQS_ERR_UNSUPPORTED
 * (nT >= 2^31, or 2^32 or more nonzeros in the rows of V), NQS_ERR_OOM, NQS_ERR_CUDA. */
int nqs_proxy_hamiltonian(nqs_problem* problem, const uint64_t* T, int64_t nV, int64_t nT,
                          const nqs_opts* opts, nqs_csr* out, nqs_stream_t stream);

/* Asymmetric mode, Sec. 2.4.1 (Eqs. asymmetric_energy, asymmetric_gradient), on T = V + P with
 * csr = nqs_proxy_hamiltonian(T, nV): E_asym = sum_{x in V} p_V(x) E_loc(x) with
 * E_loc(x) = sum_{y in T} H_xy psi_y / psi_x, i.e. sum_V psi (H_VT psi) / sum_V psi^2.
 * exact = 0: the log-derivative estimator 2 sum_V p_V(x) (E_loc(x) - E) grad ln|psi(x)| (not
 * the gradient of E_asym); exact = 1: the gradient of E_asym, which also reaches the amplitudes
 * of P: sum_{z in T} c_z grad psi_z with c_z = ((H_VT psi)_z + (H_VV psi_V)_z - 2 E psi_z) / D on
 * V and c_z = (H_PV psi_V)_z / D on P. out: device [4] = {E, N, D, max log|psi| over T}; grad
 * and psi_out as in nqs_energy_grad (over T). T need not be sorted. Stream-ordered. Errors as
 * nqs_energy_grad. */
int nqs_asym_energy_grad(nqs_problem* problem, nqs_net* net, const nqs_csr* csr,
                         const uint64_t* T, int64_t nT, int64_t nV, int exact, double* out,
                         void* grad, double* psi_out, const nqs_opts* opts, nqs_stream_t stream);

/* Post-hoc diagonalisation diagnostic E_diag = lambda_min(H_VV) (Sec. 3.5 and the Supporting
 * Information's subspace diagonalisation; Delta_opt = E_var - E_diag): Lanczos on csr (any
 * symmetric CSR, e.g. from nqs_connections) with full reorthogonalisation on the device, the
 * lowest eigenvalue of the tridiagonal by bisection. start: device [n] start vector or NULL
 * (a fixed pseudo-random vector). Stops when the lowest Ritz value changes by at most
 * tol * max(1, |lambda|) between steps, on an invariant subspace, or after max_iters steps.
 * *eigval (host) receives the value, *iters_done (host, may be NULL) the steps taken. Holds
 * (max_iters + 1) * n FP64 of scratch. Synchronises the stream every step. Errors: NQS_ERR_ARG,
 * NQS_ERR_OOM, NQS_ERR_CUDA. */
int nqs_lanczos_min(const nqs_csr* csr, int max_iters, double tol, const double* start,
                    double* eigval, int* iters_done, nqs_stream_t stream);

/* Amplitudes psi(x) of Eq. backflow_amplitude as log|psi| (device [nS] FP64) and sign (device
 * [nS] int8: +1, -1, or 0 for an exactly singular block, reported as NQS_WARN_SINGULAR).
 * Large sets are evaluated in micro-batches (opts->batch_log2, default 2^20; Sec. 3.2) so that the
 * activation memory stays bounded; dets need not be sorted. Synchronises the stream. */
int nqs_amplitudes(nqs_problem* problem, nqs_net* net, const uint64_t* dets, int64_t nS,
                   double* logabs, int8_t* sign, const nqs_opts* opts, nqs_stream_t stream);

/* Rayleigh quotient of a given vector on H_SS (Eq. variational_energy with psi injected):
 * psi device [nS] FP64; out device [3] = {E, N, D}; v device [nS] (may be NULL) = H_SS psi.
 * N and D are compensated FP64 sums. Stream-ordered, no sync. */
int nqs_energy_from_psi(const nqs_csr* csr, const double* psi, int64_t nS, double* out,
                        double* v, nqs_stream_t stream);

/* E_S and its gradient, Eqs. variational_energy and variational_gradient:
 *   psi~ = sign * exp(log|psi| - max log|psi|), v = H_SS psi~, N = psi~.v, D = psi~.psi~,
 *   E = N/D, grad = (2/D) sum_x (v_x - E psi~_x) dpsi~_x/dtheta
 * through a hand-written adjoint (Jacobi's formula with the LU inverse, then the MLP
 * backward). out: device [4] = {E, N, D, max log|psi|}. grad: device, nqs_net_num_params
 * entries laid out W1, b1, W2, b2, W3, b3 (FP64 for NQS_FP64, float for NQS_MIXED), or NULL
 * for the energy only. psi_out: device [nS] FP64 psi~ (may be NULL). Sets larger than the
 * micro-batch (opts->batch_log2) are evaluated batch by batch; the gradient then recomputes
 * each batch's activations and accumulates the batches' gradients (Sec. 3.2), so memory stays
 * bounded by the batch. Stream-ordered, no sync. csr must come from nqs_connections on the same
 * S (or nqs_proxy_hamiltonian on a target set). */
int nqs_energy_grad(nqs_problem* problem, nqs_net* net, const nqs_csr* csr, const uint64_t* dets,
                    int64_t nS, double* out, void* grad, double* psi_out, const nqs_opts* opts,
                    nqs_stream_t stream);

/* Epstein-Nesbet PT2, Eq. pt2_correction, with Psi_S = psi / sqrt(D), D = psi.psi:
 *   external = sum_{x' in C\S} c(x')^2 / (D (E - H_x'x')),  c(x') = sum_{y in S} H_x'y psi_y
 *   internal = sum_{x in S} r_x^2 / (D (E - H_xx)),         r = H_SS psi - E psi
 * C\S is generated on the device: every excitation of every y in S is emitted as
 * (key x', H_x'y psi_y) in canonical order, radix-sorted by key (stable), deduplicated, and
 * each run summed in emission order; members of S feed the internal term. The work is split
 * into hash buckets (SplitMix64 finaliser: h = mix(mix(a) ^ b), bucket = the high 32 bits of h
 * times B, shifted right by 32; B < 2^32).
 * psi: device [nS] FP64 at any scale. out: host [5] = {external, internal, number of unique
 * x' in C\S, number of emitted pairs, number of buckets used}. opts->buckets = 0 chooses the
 * bucket count: one bucket's pairs use at most half of the free device memory. bucket_partials:
 * host [2*B] (external, internal per bucket) or NULL (required with opts->buckets = 0). Sort
 * keys are 32-bit, 64-bit or two-word by 2*norb. Each bucket's emissions must stay below 2^32
 * (and fit in memory): use more buckets for larger problems.
 * With opts->eps_pt2 > 0 (Sec. 3.3: the external sum of Eq. pt2_correction runs over the
 * screened perturbative set P) only the contributions with |H_x'y psi_y| >= eps_pt2 to x' outside
 * S are emitted, found by the sorted-integral walk of nqs_hb_select; c(x') sums those, P is the
 * x' that receive at least one, and the internal term takes H_SS psi exactly from the connected
 * sets of S. Unscreened with opts->buckets = 0, when sorted buckets would traverse the connected
 * space more than eight times (their pairs do not fit in memory, or opts->chunk caps them), the
 * work runs in hashed passes instead: a pass takes a range of 256 fine buckets
 * (det_hash mod 256) sized to memory from the measured ratio of unique to emitted, accumulates
 * every emission of that range into a hash table of configurations in exact 128-bit fixed point
 * (one slot per unique x'), then sorts and reduces the unique set; out[4] then counts passes.
 * The screened runs are summed exactly in 128-bit fixed point (each term rounded
 * once to a grid far below FP64 resolution, one rounding to FP64 per x'), so c(x') does not
 * depend on the order of its terms; with opts->buckets = 0 the screened emissions are then
 * written in one traversal (appended in timing order; buffers sized from a counted sample of S
 * and enlarged once if needed) and split into counted buckets only when they do not fit in
 * memory. Synchronises the stream. Errors: NQS_ERR_ARG (also eps_pt2 < 0 or NaN),
 * NQS_ERR_OOM (a bucket too large), NQS_ERR_CUDA. */
int nqs_pt2(nqs_problem* problem, const uint64_t* dets, const double* psi, int64_t nS,
            double E_var, const nqs_opts* opts, double* out, double* bucket_partials,
            nqs_stream_t stream);

/* nqs_pt2 with H_SS at hand: hss is the library CSR of nqs_connections over the same dets (row
 * r = [diagonal, then its hits]; n_rows must equal nS). With opts->eps_pt2 > 0 the internal
 * term's off-diagonal (H_SS psi)_x is then one SpMV over hss instead of a second enumeration of
 * the connected sets of S (which at 42 orbitals costs as much as nqs_connections itself);
 * otherwise the result is the same as nqs_pt2's. hss is read only; it must stay valid until the
 * call returns. Errors: those of nqs_pt2, and NQS_ERR_ARG for a missing or mis-sized hss. */
int nqs_pt2_hss(nqs_problem* problem, const uint64_t* dets, const double* psi, int64_t nS,
                double E_var, const nqs_csr* hss, const nqs_opts* opts, double* out,
                double* bucket_partials, nqs_stream_t stream);

/* The deduplicated external set of nqs_pt2 (unscreened) for one hash bucket, for inspection
 * and testing of Eq. pt2_correction's reduction: every x' in C\S with bucket(x') = bucket (of
 * `buckets`; the bucket function of nqs_pt2), ascending by (a, b), and c(x') = sum over y in S
 * of H_x'y psi_y. Runs the same emission, sort and run reduction as nqs_pt2 for that bucket.
 * dets: device [nS][2], sorted and unique; psi: device [nS] FP64. dets_out: device [capacity][2]
 * (16-byte aligned), c_out: device [capacity]; both may be NULL with capacity 0. *n_unique
 * (host) receives the size of the set; if it exceeds capacity nothing is written and the call
 * returns NQS_ERR_ARG, so the caller can size the buffers and call again. Synchronises the
 * stream. Errors: NQS_ERR_ARG (also bucket outside 0..buckets-1), NQS_ERR_OOM, NQS_ERR_CUDA. */
int nqs_pt2_unique(nqs_problem* problem, const uint64_t* dets, const double* psi, int64_t nS,
                   int buckets, int bucket, uint64_t* dets_out, double* c_out, int64_t capacity,
                   int64_t* n_unique, nqs_stream_t stream);

/* The same set for the screened form of nqs_pt2 (opts->eps_pt2 = eps_pt2 > 0, Sec. 3.3): the x'
 * reached by at least one contribution with |H_x'y psi_y| >= eps_pt2 (psi as passed), and c(x')
 * the sum of those contributions only. Emission by the sorted-integral walk of nqs_pt2 for the
 * one bucket. Arguments, output and errors as nqs_pt2_unique; eps_pt2 <= 0 or not finite:
 * NQS_ERR_ARG. */
int nqs_pt2_unique_screened(nqs_problem* problem, const uint64_t* dets, const double* psi,
                            int64_t nS, double eps_pt2, int buckets, int bucket, uint64_t* dets_out,
                            double* c_out, int64_t capacity, int64_t* n_unique,
                            nqs_stream_t stream);

/* ---- batched evaluation of many independent problems ------------------------------------ */
typedef struct nqs_batch nqs_batch; /* opaque */

/* A batch of n independent E_S + gradient evaluations (nqs_energy_grad per problem; problems
 * may differ in norb, electron counts, |S| and network width), the "many independent
 * problems" form of the micro-batching of Sec. 3.2. All arrays have n entries and refer to
 * caller-owned objects that must outlive the batch: problems[i], nets[i] (with nets[i] created
 * on problems[i]), csrs[i] (from nqs_connections on dets[i]), dets[i] (device [nS[i]][2]),
 * outs[i] (device [4]) and grads[i] (device, or NULL for energy only). Their device addresses
 * are fixed for the batch's life (the grouped mode builds its descriptors on them once).
 * Modes (nqs_batch_set_mode):
 *   NQS_BATCH_GROUPED  each stage of the pipeline is one launch over all problems: the dense
 *                      layers as persistent tensor-core GEMMs over a (problem, tile) work list,
 *                      the LU factorisations one launch per block size, the energy stage and
 *                      the adjoint one launch each; about twenty launches per step whatever n.
 *                      Needs every net in NQS_MIXED with hidden widths divisible by 8, every
 *                      nS[i] <= 2^20, nalpha and nbeta <= 12, and grads all non-NULL or all
 *                      NULL. The default when the batch qualifies. Holds a workspace of about
 *                      (7 KB + 4 (nalpha^2 + nbeta^2) B) per configuration at width 128. With
 *                      autotuning on (nqs_set_autotune), the first run times tile widths
 *                      64/128/256 per GEMM stage and keeps the fastest.
 *   NQS_BATCH_STREAMS  nstreams side streams run the problems' own pipelines concurrently
 *                      (largest |S| first).
 * Results equal the problems' own nqs_energy_grad calls up to the order of the FP32 sums of
 * the weight gradients (the grouped GEMMs split K as the single GEMMs do at their default tile
 * widths). */
int nqs_batch_create(int n, nqs_problem* const* problems, nqs_net* const* nets,
                     const nqs_csr* csrs, const uint64_t* const* dets, const int64_t* nS,
                     double* const* outs, void* const* grads, int nstreams, nqs_batch** out);
/* Run the batch eagerly: the grouped stages on `stream`, or a fork from `stream` to one
 * pipeline per problem on the side streams and a join back. Stream-ordered; the first grouped
 * run builds the workspace and descriptors (and tunes the tile widths), synchronising. */
int nqs_batch_run(nqs_batch* batch, nqs_stream_t stream);
/* Record nqs_batch_run once into a CUDA graph (stream must not be the legacy NULL stream) and
 * instantiate it; nqs_batch_launch then replays the whole batch with one graph launch. Run
 * the batch eagerly (with autotuning on, if wanted) before capturing. */
int nqs_batch_capture(nqs_batch* batch, nqs_stream_t stream);
int nqs_batch_launch(nqs_batch* batch, nqs_stream_t stream);
int nqs_batch_destroy(nqs_batch* batch);
#define NQS_BATCH_STREAMS 0
#define NQS_BATCH_GROUPED 1
/* Select the mode; NQS_ERR_UNSUPPORTED when the batch does not qualify for the grouped mode.
 * A graph recorded in the other mode is dropped (capture again). */
int nqs_batch_set_mode(nqs_batch* batch, int mode);
/* the current mode, or NQS_ERR_ARG */
int nqs_batch_get_mode(const nqs_batch* batch);

/* GEMM tile-width autotuner (project-written): when on, the first tensor-core GEMM of each
 * shape times tile widths 64/128/256 on its stream and keeps the fastest for the process
 * (never inside stream capture). nqs_autotune_entries copies up to capacity tuned shapes
 * (M, N, K, chosen width) and returns how many there are. */
int nqs_set_autotune(int on);
int nqs_autotune_entries(int* M, int* N, int* K, int* width, int capacity);
/* Paired tensor-core GEMM (on by default): GEMMs with 256-column tiles run on clusters of two
 * SMs that share one M = 256 tcgen05.mma stream (cta_group::2), each SM staging its own 128 rows
 * of A and half of B. Off: every tile runs on one SM (M = 128). Process-wide; affects the
 * network's GEMMs and nqs_gemm_bf16, not the grouped batch GEMMs. */
int nqs_set_gemm_pairing(int on);

/* H_SS build without any device allocation (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory, such as a host framework that owns every device
 * allocation and gives the library none of its own, or an embedded solver that runs on a fixed
 * device budget). Same result as nqs_connections, written into caller-owned device buffers:
 * row_ptr [nS + 1] int64, col [capacity] int32, val [capacity] FP64. The library's scratch (hash
 * table of S, row counts, scan partials, validation flags) lives in one static device array of
 * 8 MiB, which limits nS to 65536 (larger nS returns NQS_ERR_ARG with a message in
 * nqs_last_error()). Every GPU that loads the library holds the array until process exit. The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for later calls on that device, which assumes the device's
 * primary context lives until the process exits (no cudaDeviceReset in between). *nnz (host) receives the number of nonzeros; if it
 * exceeds capacity the call returns NQS_ERR_ARG without writing col/val, so the caller can size
 * the buffers and call again. All calls share the static array, which keeps the previous
 * call's contents (what must start at zero is cleared on every call): calls that overlap on
 * the GPU race and must be serialised. validate as in nqs_opts. Synchronises the stream (the
 * number of nonzeros is read back to the host before col/val are written). */
int nqs_connections_noalloc(nqs_problem* problem, const uint64_t* dets, int64_t nS, int validate,
                            int64_t* row_ptr, int32_t* col, double* val, int64_t capacity,
                            int64_t* nnz, int64_t* n_enumerated, nqs_stream_t stream);

/* Library-owned set of configurations (device memory), ascending by (a, b). Free with
 * nqs_detset_free. */
typedef struct {
    uint64_t* dets;     /* device [n][2] */
    double* value;      /* device [n]: nqs_hb_select: max over x in S of |H_x'x| |psi_x|;
                           nqs_select: log|psi| of the kept configuration */
    int64_t* index;     /* device [n]: nqs_select: position in T; NULL for nqs_hb_select */
    int64_t n;
    int64_t n_emitted;  /* nqs_hb_select: (x, x') pairs that passed, before removing duplicates */
    int64_t n_examined; /* nqs_hb_select: candidates whose coupling was tested */
} nqs_detset;

/* Heat-bath screened perturbative set, Eq. (hb_screen) of Sec. 3.3 (Algorithm 1 step 1):
 * P = { x' not in S : max over x in S of |H_x'x psi_x| >= eps_hb }, with the product taken in
 * FP64. dets: device [nS][2], sorted and unique (checked with opts->validate); psi: device [nS]
 * FP64, the amplitudes the cutoff refers to (the caller chooses their normalisation, e.g.
 * psi / ||psi||). eps_hb >= 0 (0 keeps the whole connected set outside S). Doubles are found by
 * the sorted-integral walk with early exit of Sec. 3.3 (exact: nothing the definition keeps is
 * skipped); singles are all evaluated. The sorted integral tables are built on the first call
 * for a problem and kept until nqs_problem_destroy: 10 bytes per entry, C(norb,2) C(norb-2,2) +
 * norb^2 (norb-1)^2 entries (37 MB at norb 42, 200 MB at 64). On success *out holds a
 * library-owned set; on failure it is empty. Synchronises the stream. Errors: NQS_ERR_ARG
 * (null pointer, nS <= 0, eps_hb < 0 or NaN, misaligned dets), NQS_ERR_UNSORTED /
 * NQS_ERR_POPCOUNT (with validate), NQS_ERR_UNSUPPORTED (2^32 or more kept pairs), NQS_ERR_OOM,
 * NQS_ERR_CUDA. */
int nqs_hb_select(nqs_problem* problem, const uint64_t* dets, const double* psi, int64_t nS,
                  double eps_hb, const nqs_opts* opts, nqs_detset* out, nqs_stream_t stream);
int nqs_detset_free(nqs_detset* set);

/* Subspace selection of the outer loop, Sec. 2.4.2 (Algorithm 1 step 3: V <- Selector(T, K,
 * key = |psi|)). T: device [n][2] configurations (any order, no repeats: checked with
 * opts->validate); logabs: device [n] log|psi| (as nqs_amplitudes returns it; -inf for psi = 0;
 * NaN or +inf is an error). Ranking: log|psi| descending, ties by ascending (a, b). With
 * w = exp(2 (log|psi| - max log|psi|)) and D = sum of w over T, the kept prefix is
 *   NQS_SELECT_TOPK       the first min(K, n) (param unused);
 *   NQS_SELECT_MASS       the shortest prefix whose sum of w reaches param * D
 *                         (0 <= param <= 1; all of T if rounding keeps it below);
 *   NQS_SELECT_THRESHOLD  every x with w_x / D > param (param >= 0; K unused).
 * *out receives the kept configurations ascending by key (the next S), their log|psi| and their
 * positions in T. Sums are FP64 in a fixed device order: at the boundary of the mass and
 * threshold protocols the count can differ from a serial sum by the configurations whose
 * running mass or weight lies within rounding of the cutoff. Synchronises the stream. Errors:
 * NQS_ERR_ARG, NQS_ERR_UNSORTED (repeated configuration, with validate), NQS_ERR_OOM,
 * NQS_ERR_CUDA. */
#define NQS_SELECT_TOPK 0
#define NQS_SELECT_MASS 1
#define NQS_SELECT_THRESHOLD 2
int nqs_select(nqs_problem* problem, const uint64_t* T, const double* logabs, int64_t n, int mode,
               int64_t K, double param, const nqs_opts* opts, nqs_detset* out,
               nqs_stream_t stream);

/* Plain library GEMM on the tensor cores used by the backflow network (not a step of the
 * paper's method; exposed for testing and reuse): C[m][n] = sum_k A[m][k] B[n][k] with A
 * [M][lda] and B [N][ldb] bfloat16, k contiguous (lda, ldb multiples of 8, 16-byte aligned
 * bases), C [M][ldc] float, FP32 accumulation. err_flag (device int, may be NULL) is set to 1
 * if a bounded pipeline wait timed out. Stream-ordered, no sync. Returns NQS_ERR_UNSUPPORTED
 * for strides the tensor-memory-access unit cannot take. */
int nqs_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                  float* C, int64_t ldc, int* err_flag, nqs_stream_t stream);
/* The same GEMM with either operand stored MN-major (the layout the weight gradients of the
 * network read: row-major activations, no transposed copy): a_mn = 1 means A[m][k] is at
 * A[k * lda + m] (A is [K][lda], m contiguous, lda >= M); b_mn = 1 means B[n][k] is at
 * B[k * ldb + n]. a_mn = b_mn = 0 is nqs_gemm_bf16. Alignment rules and errors as above. */
int nqs_gemm_bf16_ex(const void* A, int64_t lda, int a_mn, const void* B, int64_t ldb, int b_mn,
                     int M, int N, int K, float* C, int64_t ldc, int* err_flag,
                     nqs_stream_t stream);

/* ---- failure detection and memory accounting (not steps of the method) ------------------ */
/* Check of the timeout path: one device thread waits, with the same bounded mbarrier wait as
 * the tensor-core GEMM pipeline, on a barrier that nothing completes; the wait gives up after
 * limit_cycles SM clocks (1 .. 4e9; the pipeline's own limit is 4e9, about 2 s) and reports
 * through the problem's error word exactly as a timed-out pipeline does. Returns
 * NQS_ERR_TIMEOUT (the expected result) and clears the word; the CUDA context stays usable.
 * Synchronises the stream. Errors: NQS_ERR_ARG, NQS_ERR_CUDA. */
int nqs_wait_probe(nqs_problem* problem, int64_t limit_cycles, nqs_stream_t stream);
/* Cap on the problem's stream-ordered scratch pool: a scratch request that would take the
 * pool's bytes in use above `bytes` fails and the call returns NQS_ERR_OOM, with every
 * scratch block it took returned to the pool. 0 removes the cap. Errors: NQS_ERR_ARG. */
int nqs_set_scratch_limit(nqs_problem* problem, int64_t bytes);
/* Bytes of the problem's scratch pool in use (scratch of running calls and library-owned CSRs)
 * and reserved from the device (kept between calls). Errors: NQS_ERR_ARG, NQS_ERR_CUDA. */
int nqs_pool_usage(nqs_problem* problem, int64_t* used, int64_t* reserved);

/* Optional per-kernel timing for benchmarks (not part of the method): when enabled, the
 * library brackets its main kernel launches with CUDA events recorded on the launching stream.
 * nqs_profile_read synchronises those events and returns the summed milliseconds and the
 * launch count of one kernel family: "conn_count", "conn_fill", "pt2_count", "pt2_emit",
 * "rs_hist", "rs_scatter", "seg_reduce", "gemm", "lu", "spmv", "layer1", "unique_terms",
 * "heads", "scan", "hb_select", "select". Process-wide state;
 * not thread safe. */
int nqs_profile_enable(int on);
int nqs_profile_reset(void);
int nqs_profile_read(const char* kernel, double* total_ms, int64_t* launches);
/* number of kernels this library has launched in this process so far */
int64_t nqs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
