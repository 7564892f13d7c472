/*
 * sfci.h -- C ABI of the GB300 sparse-FCI sigma = H psi library (libsfci.so).
 *
 * The method is Sparse Full Configuration Interaction (L. Wang, arXiv
 * 2312.01846): a Lanczos-like solver whose basis vectors are truncated to the
 * N_d largest-magnitude determinants (Sec. 2.1, Eqs. 10-11), built on a sparse
 * Hamiltonian x sparse vector product whose intermediate elements are
 * generated on the fly and merged by a consecutive-integer index of the
 * determinants (Sec. 2.2, Eq. 12).
 *
 * Conventions used by every call:
 *  - A determinant is a pair of spin strings (alpha, beta), each a uint64 with
 *    bit p set when spatial orbital p (0-based) is occupied; n <= 64.
 *  - A spin string's index is Eq. 12, h = sum_i C(chi_i - 1, i) with chi_i the
 *    i-th occupied orbital counted from 1 (the colex rank).  A determinant's
 *    index ("rank") is alpha-major: rank = h(alpha) * C(n, n_beta) + h(beta),
 *    a bijection onto [0, dim), dim = C(n, n_alpha) C(n, n_beta) (Sec. 3 buckets
 *    on the spin-up string only; alpha-major ranks make those buckets
 *    contiguous rank ranges).
 *  - A sparse vector is two arrays: uint64 rank[m] strictly ascending and
 *    double coef[m] ("2-tuples (i, alpha_i)", Sec. 2.2).
 *  - Integrals: h[p*n+q] = h_pq and g[((p*n+q)*n+r)*n+s] = (pq|rs) in
 *    chemists' notation, real orbitals, 8-fold symmetric, float64, row-major.
 *  - H = e_core + sum_pq h_pq sum_s a+_ps a_qs
 *          + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs.
 *    Determinants are ordered products of creators, alpha orbitals ascending
 *    then beta ascending; that fixes the signs of sigma's entries.
 *  - Pointers documented "device" must be CUDA device (or managed) memory on
 *    the current device; "host" pointers are ordinary host memory.  `stream`
 *    is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    All work of a call is ordered on that stream.
 *  - Every call returns an sfci_status; none throws or aborts.  On failure
 *    sfci_last_error() gives a thread-local message.  Calls that return a
 *    count to the host synchronise `stream`.
 *  - Ownership: the caller owns every vector, output and workspace buffer;
 *    the library owns handles and the device copies of the integrals.
 */
#ifndef SFCI_H
#define SFCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sfci_status {
    SFCI_OK = 0,
    SFCI_E_INVALID = 1,  /* bad argument, unsorted input, rank >= dim, ...    */
    SFCI_E_CAPACITY = 2, /* an output or workspace is too small; see the call */
    SFCI_E_OVERFLOW = 3, /* n > 64 or dim does not fit below 2^64 - 1         */
    SFCI_E_CUDA = 4,     /* a CUDA runtime call failed                         */
    SFCI_E_TIMEOUT = 5,  /* a bounded device wait ran out                      */
    SFCI_E_NOMEM = 6     /* device or host allocation failed                   */
} sfci_status;

/* Static, human-readable name of a status code. */
const char *sfci_status_string(int status);
/* Detail of the last failure on the calling thread ("" if none). */
const char *sfci_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int sfci_version(void);
/* Number of CUDA kernels the library has launched in this process so far
 * (a diagnostic: the difference across a region counts its launches). */
int64_t sfci_kernel_launches(void);

/* ------------------------------------------------------------- system */

typedef struct sfci_system sfci_system; /* opaque */

/* sfci_system_create flags */
/* Off-diagonal Slater-Condon elements (singles and doubles) from float32
 * copies of h and g, with float32 sums for the singles.  The diagonal, the
 * product element * c_D, the accumulation of sigma, the dots and the
 * eigensolve stay float64.  Not in the paper (which works in float64): a
 * precision option whose energy error against the float64 path is measured
 * per result, not bounded a priori. */
#define SFCI_FP32_ELEMENTS 1u

/* Copy the integrals (host pointers; h: n*n, g: n^4 float64) to the current
 * device and build the binomial table C(b, m) used by Eq. 12.  n in [1, 64],
 * 0 <= n_alpha, n_beta <= n.  Returns SFCI_E_OVERFLOW when dim >= 2^64 - 1,
 * SFCI_E_INVALID for bad counts or unknown flag bits.  flags: 0 or
 * SFCI_FP32_ELEMENTS. */
sfci_status sfci_system_create(sfci_system **out, int n_orb, int n_alpha, int n_beta,
                               const double *h_host, const double *g_host, double e_core,
                               uint32_t flags);
sfci_status sfci_system_destroy(sfci_system *sys);
/* dim = C(n, n_alpha) C(n, n_beta). */
sfci_status sfci_dim(const sfci_system *sys, uint64_t *dim);
/* Determinants connected to one determinant by single and double
 * excitations: na va + nb vb + C(na,2)C(va,2) + C(nb,2)C(vb,2) + na va nb vb
 * (v = n - n_electrons).  Intermediate elements per input entry = this + 1. */
sfci_status sfci_n_connected(const sfci_system *sys, int64_t *n_conn);

/* ---------------------------------------------------------- Eq. 12 */

/* rank[i] = alpha-major index of (alpha[i], beta[i])  (Eq. 12).  Device
 * pointers, count entries.  SFCI_E_INVALID if any string has the wrong
 * electron count or bits at or above n (those ranks are set to UINT64_MAX).
 * Synchronises the stream. */
sfci_status sfci_rank(const sfci_system *sys, const uint64_t *alpha, const uint64_t *beta,
                      uint64_t *rank, int64_t count, void *stream);
/* Inverse of sfci_rank (greedy inverse of Eq. 12).  SFCI_E_INVALID if some
 * rank >= dim (those strings are set to 0).  Synchronises the stream. */
sfci_status sfci_unrank(const sfci_system *sys, const uint64_t *rank, uint64_t *alpha,
                        uint64_t *beta, int64_t count, void *stream);

/* ---------------------------------------------------------- sigma = H psi */

/* Workspace (bytes, device) that sfci_sigma needs for n_in input entries and
 * room for out_cap output entries.  It holds an open-addressing table of
 * 2^ceil(log2(2 out_cap)) slots (at least 1024; 32 bytes each with the exact
 * sums) plus sort buffers. */
sfci_status sfci_sigma_workspace_bytes(const sfci_system *sys, int64_t n_in, int64_t out_cap,
                                       size_t *bytes);

/* sigma = H psi (Sec. 2.2).  For every input entry (D, c_D) the library
 * enumerates D and all its single and double excitations D', evaluates the
 * Slater-Condon element <D'|H|D>, and adds the intermediate element
 * <D'|H|D> c_D into the entry of rank(D'); exactly-zero products are not
 * generated.  Entries that received at least one non-zero element and whose
 * |sum| >= eps_screen (eps_screen <= 0: no screen; the paper's epsilon of
 * Sec. 3) are written to out_rank/out_coef (device) ascending by rank, and
 * their count to *n_out (host).
 * in_rank/in_coef: device, n_in entries, ranks strictly ascending and < dim.
 * Returns SFCI_E_CAPACITY if more than out_cap entries result: then *n_out is
 * the exact count when it is at most the table's slot count, otherwise a lower
 * bound (retry with a larger out_cap).  SFCI_E_CAPACITY also when ws_bytes is
 * below sfci_sigma_workspace_bytes.  No allocation; synchronises the stream.
 * Each entry is summed exactly (128-bit fixed point in units of 2^-S, S set
 * from (n_conn + 1) max|h, g element| max|c_D| so that no sum leaves the
 * range) and rounded once to float64: the result does not depend on the order
 * of the adds and is the same on every run.  SFCI_E_INVALID for non-finite
 * coefficients. */
sfci_status sfci_sigma(const sfci_system *sys, const uint64_t *in_rank, const double *in_coef,
                       int64_t n_in, double eps_screen, uint64_t *out_rank, double *out_coef,
                       int64_t out_cap, int64_t *n_out, void *workspace, size_t ws_bytes,
                       void *stream);

/* ---------------------------------------------------------- Eq. 11 */

sfci_status sfci_truncate_topk_workspace_bytes(int64_t n, int64_t k, size_t *bytes);

/* Truncation of Eq. 11: keep the min(k, #non-zero) entries of largest |coef|;
 * among equal |coef| the smaller rank wins; exact zeros are never kept.  With
 * normalize != 0 the kept coefficients are divided by their 2-norm
 * sqrt(sum c^2).  rank/coef: device, n entries, ranks unique (any order).
 * Output (device, room for k entries) ascending by rank; *n_out (host) = kept
 * count.  Selection is exact: decided on the bit patterns of |coef| and rank.
 * No allocation; synchronises the stream. */
sfci_status sfci_truncate_topk(const uint64_t *rank, const double *coef, int64_t n, int64_t k,
                               int normalize, uint64_t *out_rank, double *out_coef,
                               int64_t *n_out, void *workspace, size_t ws_bytes, void *stream);

/* sfci_truncate_topk without a workspace, for callers that cannot allocate
 * device memory (a host framework that owns all of it through its own pool, a
 * plugin given a fixed budget, a loop that must not reach the allocator).
 * The paper has no counterpart: this is a library convenience.  Same inputs,
 * outputs, selection and errors as sfci_truncate_topk.
 *   - Scratch: one fixed 20 MiB device array inside the library (one per
 *     device), so k <= 1048576; a larger k returns SFCI_E_CAPACITY and the
 *     reason in sfci_last_error().  n is not limited by the scratch.
 *   - The call allocates nothing, neither does any kernel it launches.  It
 *     clears the parts of the scratch that must start at zero itself.
 *   - The first call on each device looks up the scratch's device address
 *     (with that device current) and caches it; make that first call before
 *     any stream capture.  The cache lives as long as the process and does
 *     not survive a reset of the device (cudaDeviceReset or a new primary
 *     context): after one, do not call this entry point again in that
 *     process.
 *   - All calls on one device share the scratch: calls that overlap in time
 *     (other threads, other streams) race and corrupt each other's results.
 *     Serialise them.
 *   - Synchronises the stream. */
sfci_status sfci_truncate_topk_noalloc(const uint64_t *rank, const double *coef, int64_t n,
                                       int64_t k, int normalize, uint64_t *out_rank,
                                       double *out_coef, int64_t *n_out, void *stream);

/* ---------------------------------------------------------- SFCI Lanczos */

/* sfci_params.flags */
/* A test setting for the automatic bucket size (bucket_elems = 0): every
 * sigma first tries 2048-element merge buckets in 1024-slot tables, which
 * cannot hold a bucket with more than 1024 distinct entries; such a sigma is
 * redone with the normal 1024-element buckets (info->bucket_redo), with the
 * same result.  Exercises the fallback that a crowded 2048-element bucket
 * takes in normal runs; slower. */
#define SFCI_LZ_FALLBACK_STRESS 1u

typedef struct sfci_params {
    int64_t n_keep;         /* N_d: entries kept per basis vector (Eq. 11)          */
    int64_t table_capacity; /* slots of sigma's hash table; 0 = sized automatically */
    double eps_screen;      /* drop |sigma_k| < eps_screen before the dots (Sec. 3) */
    double conv_tol;        /* halt when E(n-1) - E(n) < conv_tol (Sec. 2.1); <= 0 off */
    int32_t n_lanczos;      /* N_L: basis vectors per cycle, w_0 included (Sec. 2.1) */
    int32_t max_iter;       /* the step that reaches this sigma count ends its cycle; <= 0 off */
    uint32_t flags;         /* 0 or SFCI_LZ_FALLBACK_STRESS                           */
    int32_t bucket_elems;   /* intermediate elements per merge bucket; 0 = automatic:
                               1024, or 2048 once the previous sigma had at least
                               1.5 elements per distinct entry (a table overflow
                               then redoes that sigma with 1024 and raises that
                               level to 1.25 times the repetition that failed)    */
    int64_t mem_budget;     /* device bytes this solver's sigma buffers may take;
                               0 = 85 % of what is free (one solver per device)   */
    int32_t emit_warps;     /* warps per CTA of the element generator (1..8); 0 = 8 */
    int32_t ovf_max_log2;   /* the overflow list (elements past their merge bucket's
                               region) holds at most 2^ovf_max_log2 entries;
                               0 = sized from free memory.  A pass whose overflow
                               does not fit is split into pieces, or sigma is
                               redone with a longer list (up to this limit);
                               SFCI_E_CAPACITY when no attempt fits            */
    double eps_element;     /* heat-bath style selection (the outlook of Sec. 4):
                               intermediate elements with |<D'|H|D> c_D| <
                               eps_element are not generated, whole excitation
                               classes skipped by integral bounds; 0 = exact sigma */
} sfci_params;

typedef struct sfci_step_info {
    int32_t iter;      /* sigma applications so far, this one included (N_I)        */
    int32_t cycle;     /* cycle (restart) index of this step                        */
    int32_t index;     /* i: position of this step's input w_i within its cycle     */
    int32_t cycle_end; /* 1: this step solved T x = lambda S x and restarted        */
    int32_t converged; /* 1: the halting test passed at this cycle end              */
    int32_t breakdown; /* 1: u vanished (||u|| < 1e-14 |a_i|) and the cycle ended     */
    double lambda_min; /* lowest root of T x = lambda S x (valid when cycle_end)    */
    double a;          /* a_i = <w_i|sigma_i>                                       */
    double b;          /* b_i = <w_{i-1}|sigma_i> (0 for i = 0)                      */
    double u_norm;     /* ||u_{i+1}|| before truncation (0 at a cycle end)          */
    double t00;        /* <w_0|H|w_0> of this cycle                                 */
    int64_t n_in;      /* entries of w_i                                            */
    int64_t n_sigma;   /* entries of sigma_i after the screen                       */
    int64_t n_kept;    /* entries of the next basis vector                          */
    int64_t n_elements;/* intermediate elements enumerated for sigma_i              */
    int64_t n_psi;     /* non-zero entries of Psi = sum_j x_j w_j (cycle end)         */
    double ms_sigma;   /* device time of the sigma stage (CUDA events)              */
    double ms_step;    /* device time of the whole step                             */
    double ms_emit;    /* of ms_sigma: the emit kernel (all passes)                 */
    double ms_merge;   /* of ms_sigma: overflow sort + merge kernel (all passes)    */
    double ms_plan;    /* wall time of the bucket plan (row weights, device plan,
                          pass cuts) and of sizing the buffers                  */
    double ms_topk;    /* device time of the truncation (u entries, top-k, sort)    */
    int32_t n_passes;  /* passes over the sources that sigma needed (memory bound, plus
                          passes split because their overflow outgrew the list) */
    int32_t n_buckets_log2; /* ceil(log2(merge buckets))                            */
    double tau;        /* stream threshold of the accepted attempt (entries of sigma
                          below it were not written out; see sfci_lanczos_step)  */
    double cut;        /* |coef| of the N_d-th kept entry of u (0 if fewer kept)    */
    int32_t redo;      /* sigma recomputed because tau hid part of the N_d largest  */
    int32_t bucket_redo; /* sigma recomputed with 1024-element buckets because a
                            2048-element bucket outgrew its table (automatic size) */
    double pass_budget_gb; /* device memory one pass's element regions may use (GB) */
    double regions_gb;     /* element regions of all buckets (GB): passes ~ this/budget */
    double free_gb;        /* free device memory the plan saw, besides the solver's
                              element, stream and overflow buffers (GB)              */
    int64_t n_overflow;    /* most elements any pass sent past their bucket's region  */
    double ms_alloc;       /* of ms_plan: device buffer (re)allocation               */
    int64_t n_emitted;     /* intermediate elements generated for sigma_i and merged:
                              the non-zero products of n_elements                */
    int64_t n_alpha_runs;  /* runs of consecutive entries of w_i that share alpha
                              (0: not counted, hash mode)                         */
} sfci_step_info;

typedef struct sfci_lanczos sfci_lanczos; /* opaque; owns w_0..w_{N_L-1}, T, S, table */

/* Start a solver from a trial vector (device pointers, ranks strictly
 * ascending; the paper starts from one determinant, Sec. 3).  The trial
 * vector is truncated to n_keep and normalised to become w_0.  Allocates the
 * solver's device memory; the system must outlive the solver. */
sfci_status sfci_lanczos_create(sfci_lanczos **out, const sfci_system *sys,
                                const sfci_params *params, const uint64_t *init_rank,
                                const double *init_coef, int64_t n_init, void *stream);
/* One sigma application (one of the paper's N_I iterations):
 *   sigma_i = H w_i (screened); T_ji = <w_j|sigma_i>, S_ji = <w_j|w_i> for j <= i;
 *   then either w_{i+1} = normalise(top_{N_d}(sigma_i - a_i w_i - b_i w_{i-1}))
 *   (Eqs. 10-11), or, at the cycle's last vector, the lowest root of
 *   T x = lambda S x, Psi = sum_j x_j w_j, and w_0 = normalise(top_{N_d}(Psi)).
 * info (host) receives the step's scalars.  Synchronises the solver's stream.
 * Only the entries of u that can be among the N_d largest leave the merge:
 * those with |u| >= tau, tau predicted from earlier cuts.  The step then checks
 * that the N_d-th kept |u| is >= tau; if not, it recomputes sigma with the
 * exact threshold read off a magnitude histogram of this attempt (info->redo),
 * so the kept set is the exact top-N_d of Eq. 11 either way.
 * SFCI_E_CAPACITY only if sigma's buffers cannot grow in device memory.
 * Observability: when the environment variable SFCI_STEP_LOG names a file,
 * every step appends one JSON line to it (iteration, cycle, lambda, a, b,
 * ||u||, entries kept, elements, stage times and the sigma stage's rate
 * under 32 bytes per element); the stages are also marked as NVTX ranges
 * for a profiler's timeline. */
sfci_status sfci_lanczos_step(sfci_lanczos *lz, sfci_step_info *info);
/* Restart the solver from a new trial vector (device pointers, ranks strictly
 * ascending): it is truncated to n_keep and normalised into w_0, and a new
 * cycle begins (T, S and the halting history are cleared).  Lets a caller
 * stream vectors through the solver without re-creating it. */
sfci_status sfci_lanczos_load(sfci_lanczos *lz, const uint64_t *rank, const double *coef,
                              int64_t n);
/* Overwrite the current input vector (the w_i the next step will use) with a
 * caller's copy, keeping the cycle's T, S and w_0 .. w_{i-1}: resuming a run
 * whose vectors live elsewhere (a host checkpoint, another process).  The
 * vector (device pointers, ranks strictly ascending, 1 <= n <= n_keep) is
 * taken as it is: it should be the w_i that sfci_lanczos_vector returned,
 * or the cycle's T and S no longer describe the basis.  SFCI_E_CAPACITY if
 * n > n_keep.  Synchronises the solver's stream. */
sfci_status sfci_lanczos_set_input(sfci_lanczos *lz, const uint64_t *rank, const double *coef,
                                   int64_t n);
/* Copy the current input vector (the w_i the next step will use) to device
 * buffers with room for cap entries; *n (host) = its length. */
sfci_status sfci_lanczos_vector(const sfci_lanczos *lz, uint64_t *rank, double *coef,
                                int64_t cap, int64_t *n);
/* T and S of the current cycle so far (host, n_lanczos^2 each, row-major,
 * upper triangle j <= i filled).  Right after a step that ended a cycle
 * (info->cycle_end = 1), the T and S that step solved. */
sfci_status sfci_lanczos_matrices(const sfci_lanczos *lz, double *T, double *S);
sfci_status sfci_lanczos_destroy(sfci_lanczos *lz);

/* ---------------------------------------------------------- batched scan */

/* Many independent SFCI problems advanced together, e.g. a scan along a
 * geometry-like parameter with uneven orbital counts, electron counts and
 * N_d.  Not in the paper (which solves one system at a time): a runtime for
 * running its method on many systems at once on one GPU.
 *   count instances; systems[i] (all on one device), params[i] and the trial
 *   vector (init_rank[i], init_coef[i], n_init[i], device pointers, ranks
 *   strictly ascending) as for sfci_lanczos_create.  params[i].mem_budget = 0
 *   gives instance i a share of 80 % of the free device memory in proportion
 *   to N_d (n_conn + 1).  workers = host threads (0: min(count, 8)).
 * Each instance runs on its own non-blocking stream; the scan owns the
 * solvers and streams.  The systems must outlive the scan. */
typedef struct sfci_scan sfci_scan;
sfci_status sfci_scan_create(sfci_scan **out, int32_t count, const sfci_system *const *systems,
                             const sfci_params *params, const uint64_t *const *init_rank,
                             const double *const *init_coef, const int64_t *n_init,
                             int32_t workers);
/* One sfci_lanczos_step of every instance (Sec. 2.1, Eqs. 10-11 as there),
 * run concurrently: worker threads take instances from a queue, largest
 * expected work first.  infos (host, count entries) receives each instance's
 * step information.  Returns the first failing instance's status (its index
 * in sfci_last_error()); the other instances still completed their step. */
sfci_status sfci_scan_step(sfci_scan *scan, sfci_step_info *infos);
/* The solver of instance i (owned by the scan), for sfci_lanczos_vector and
 * sfci_lanczos_matrices.  Do not step or destroy it directly. */
sfci_status sfci_scan_solver(sfci_scan *scan, int32_t i, sfci_lanczos **out);
sfci_status sfci_scan_destroy(sfci_scan *scan);

/* ---------------------------------------------------------- density matrices */

/* Workspace (bytes, device) for sfci_rdm12 on a vector of n entries. */
sfci_status sfci_rdm12_workspace_bytes(const sfci_system *sys, int64_t n, size_t *bytes);

/* Spin-summed one- and two-particle density matrices of psi (not normalised),
 * produced by the sigma excitation generator (every D' in {D} and the single
 * and double excitations of D that psi holds):
 *   rdm1[p*n+q]             = sum_s   <psi| a+_ps a_qs |psi>
 *   rdm2[((p*n+q)*n+r)*n+s] = sum_st  <psi| a+_ps a+_rt a_st a_qs |psi>
 * so that <psi|H|psi> = e_core <psi|psi> + sum h rdm1 + 1/2 sum (pq|rs) rdm2, and
 * for fixed psi dE/dh = rdm1 / <psi|psi>, dE/d(pq|rs) = rdm2 / (2 <psi|psi>).
 * These gradients of the Rayleigh energy are the adjoint the paper does not
 * have (its method stops at the energy, Sec. 2.1).
 * rank/coef: device, n entries, ranks strictly ascending and < dim.  rdm1
 * (n^2) and rdm2 (n^4) are device float64 outputs (overwritten); *norm2 (host,
 * may be NULL) receives <psi|psi>.  Accumulates with atomic adds (rounding order
 * not fixed).  No allocation; synchronises the stream. */
sfci_status sfci_rdm12(const sfci_system *sys, const uint64_t *rank, const double *coef, int64_t n,
                       double *rdm1, double *rdm2, double *norm2, void *workspace,
                       size_t ws_bytes, void *stream);

/* The Rayleigh energy of psi from its density matrices and a set of integrals:
 *   *energy = e_core + (sum_pq h_pq rdm1_pq + 1/2 sum_pqrs g_pqrs rdm2_pqrs) / norm2
 * (the expectation value of H in the form given above; Sec. 2.1 takes the
 * ground-state energy as this Rayleigh quotient).  rdm1, rdm2 as written by
 * sfci_rdm12 and norm2 = <psi|psi> from it; h (n^2) and g (n^4) device float64
 * in the layout of sfci_system_create, so the integrals may differ from the
 * system's (the energy as a function of h and g for a fixed psi).  workspace:
 * device, at least 2456 bytes.  Sums in a fixed order (repeatable).
 * Synchronises the stream. */
sfci_status sfci_rdm_energy(int n_orb, const double *rdm1, const double *rdm2, double norm2,
                            const double *h, const double *g, double e_core, double *energy,
                            void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------- test exports */

/* Every intermediate element of the given entries, unscaled: for input entry
 * s (device rank[s]) and each of its n_conn + 1 targets D' (D itself first),
 * src[s*(n_conn+1)+e] = s, tgt[...] = rank(D'), elem[...] = <D'|H|D>.
 * Device outputs with room for cap entries; *n_out (host) = n*(n_conn+1).
 * Synchronises the stream. */
sfci_status sfci_debug_excitations(const sfci_system *sys, const uint64_t *rank, int64_t n,
                                   int64_t *src, uint64_t *tgt, double *elem, int64_t cap,
                                   int64_t *n_out, void *stream);

/* Diagnostic: the rate (lane operations per second) of one SM pipe operation
 * that bounds the sigma kernels, measured alone on the current device with
 * enough independent work per thread to fill the pipe.  kind: 0 float64
 * fused multiply-add, 1 float64 add, 2 float64 multiply, 3 float32 fused
 * multiply-add, 4 64-bit integer multiply-add, 5 64-bit integer atomic add on
 * shared memory, 6 32-bit integer atomic add on shared memory, 7 64-bit
 * compare-and-swap on shared memory, 8 float32 atomic add on shared memory.
 * iters in [1, 2^30] loop trips per thread (8 operations each for kinds 0-4,
 * 2 for 5-8); workspace: 8 bytes of
 * device memory.  Not part of the method: it gives the issue-rate ceilings
 * against which the kernels' counters are read.  Synchronises the stream. */
sfci_status sfci_debug_pipe_rate(int kind, int64_t iters, void *workspace, double *ops_per_s,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SFCI_H */
