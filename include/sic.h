/*
 * libsic -- sparse inverse Cholesky factors of dense kernel matrices by greedy
 * conditional selection, on one GB300 (sm_103a).
 *
 * Method: Huan, Guinness, Katzfuss, Owhadi, Schaefer, "Sparse inverse Cholesky
 * factorization of dense kernel matrices by greedy conditional selection".
 * For each column i of the factor L (L L^T ~ Theta^{-1}, lower triangular in a
 * reverse-maximin elimination order), candidates j are scored by the reduction of
 * the target's conditional variance cov_j^2 / var_j (Section 3.1, eq. obj_gp), the
 * best is selected, the partial Cholesky factor gains the column
 * u = (Theta[:, q] - F F[q, :]^T) / sqrt(var_q) (eq. cond_select, Appendix B.1), and
 * after k picks the column is filled with the KL-optimal values
 * L_{s,i} = Theta_{s,s}^{-1} e_1 / sqrt(e_1^T Theta_{s,s}^{-1} e_1) (eq. L_col).
 * Supernodes share one selection among m consecutive targets and score candidates
 * by the log-determinant change of the targets' conditional covariance
 * (Section 5.2, eq. greedy_mult).
 *
 * Conventions shared by every entry point
 *  - Points are row-major FP64, n x dim (dim = 1, 2 or 3), already in elimination
 *    order for the selection and fill calls: row p is the point at position p.
 *  - Pointers marked [device] are device pointers owned by the caller; the library
 *    never frees or retains them.  Pointers marked [host] are host memory.
 *  - Every device call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream).  Argument errors are returned at once;
 *    errors found by a kernel (a non-positive-definite pivot, a bound exceeded) are
 *    recorded in the handle and returned by sic_sync().
 *  - `ws` / `ws_bytes` is caller-owned device scratch sized by the matching
 *    *_workspace call; too small a workspace returns SIC_ERR_INVALID.
 *  - No call falls back to the CPU: without a usable GPU they return SIC_ERR_CUDA.
 *  - The factor is CSC: col_ptr[n+1] (int64), row_idx (int32 positions), val (FP64).
 *    Each column lists its diagonal first, then the other rows in ascending order.
 */
#ifndef SIC_H
#define SIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIC_OK = 0,
    SIC_ERR_INVALID = 1,     /* bad argument: size, pointer, range */
    SIC_ERR_NOT_PD = 2,      /* a kernel met a non-positive pivot (see sic_last_error_unit) */
    SIC_ERR_CUDA = 3,        /* a CUDA runtime call failed (no device, launch failure, ...) */
    SIC_ERR_OOM = 4,         /* the handle could not allocate its own small state */
    SIC_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    SIC_ERR_UNSUPPORTED = 6  /* valid request outside the compiled size envelope */
} sic_status;

/* Matern kernel (Section 2; parameterised by sqrt(2 nu) r / length_scale).
 * Theta_{ab} = variance * M_nu(|x_a - x_b|) for a != b, plus `nugget` on the diagonal. */
typedef struct {
    int32_t dim;          /* 1, 2 or 3 */
    int32_t nu_x2;        /* twice the smoothness: 1, 3 or 5 (nu = 1/2, 3/2, 5/2) */
    double length_scale;  /* > 0 */
    double variance;      /* > 0 */
    double nugget;        /* >= 0 */
} sic_kernel;

/* Arithmetic of the selection kernels.  The fill and the KL sum are always FP64.
 * SIC_FP64 evaluates the kernel with a table-driven exp and Newton square roots (about
 * 2 ulp); SIC_FP32_MIXED uses the hardware's approximate reciprocal, reciprocal square
 * root and exp (a few ulp of FP32), far below the FP32 state's own resolution. */
typedef enum {
    SIC_FP64 = 0,        /* scores, partial factor and downdates in FP64 */
    SIC_FP32_MIXED = 1   /* kernel entries, partial factor and downdates in FP32 */
} sic_precision;

typedef enum { SIC_OP_L = 0, SIC_OP_LT = 1, SIC_OP_LLT = 2 } sic_op;

typedef struct sic_handle sic_handle;

/* ---------------------------------------------------------------- handle -- */

/* Binds a handle to CUDA device `device` and allocates its status word.
 * Returns SIC_ERR_CUDA if the device cannot be used. */
sic_status sic_create(sic_handle** h, int device);
void sic_destroy(sic_handle* h);

/* Waits for `stream`, then returns (and clears) the first error a kernel recorded
 * since the last sic_sync, or SIC_ERR_CUDA if the stream itself failed. */
sic_status sic_sync(sic_handle* h, void* stream);

/* Column (or group) index attached to the error last returned by sic_sync, or -1. */
int64_t sic_last_error_unit(sic_handle* h);

const char* sic_status_string(sic_status s);

/* Exhaustion floor used by the selections: a candidate whose conditional variance
 * falls below it is never picked.  0.5 * nugget, or 1e-14 * variance without nugget
 * (every exact conditional variance is at least the nugget). */
double sic_exhaustion_floor(const sic_kernel* kp);

/* ------------------------------------------------- input preparation [host] -- */

/* Reverse-maximin ordering (Section 2.2, eq. maximin).  The last position holds
 * point 0; each earlier position holds the unplaced point farthest (squared FP64
 * Euclidean distance, ties to the lowest point index) from the points already
 * placed.  order[p] = index of the point at position p; ell2[p] = squared distance
 * from it to the points after it (INFINITY at p = n-1).  All buffers [host].
 * n_threads <= 0 means all hardware threads. */
sic_status sic_prep_maximin(const double* pts, int64_t n, int32_t dim, int64_t* order, double* ell2,
                            int32_t n_threads);

/* Candidate lists of single columns (Section 4): for each position i the n_cand
 * points at positions > i nearest to point i, sorted by (squared distance,
 * position); fewer near the end of the ordering.  cand_ptr[n+1] receives CSR
 * offsets; cand_idx must hold n * n_cand entries.  pts in elimination order. [host] */
sic_status sic_prep_candidates_columns(const double* pts, int64_t n, int32_t dim, int32_t n_cand,
                                       int64_t* cand_ptr, int32_t* cand_idx, int32_t n_threads);

/* Supernodes (Section 6.1 grouping rule): the first position i not yet grouped opens a
 * group with the not-yet-grouped j among its K nearest later points (distance order)
 * with ell2_j <= lambda^2 ell2_i, at most mmax members; then each group smaller than
 * mmin is merged into the group formed just before it if the union has at most mmax
 * members.  members[n] lists old positions in the renumbered order (group after group,
 * ascending within a group); grp_ptr[n+1] receives the group offsets and *n_grp the
 * group count.  [host] */
sic_status sic_prep_groups(const double* pts, const double* ell2, int64_t n, int32_t dim, int32_t K,
                           double lambda, int32_t mmin, int32_t mmax, int64_t* members, int64_t* grp_ptr,
                           int64_t* n_grp, int32_t n_threads);

/* Candidate lists of groups: for group g (positions grp_ptr[g] .. grp_ptr[g+1]-1)
 * the n_cand points at positions >= grp_ptr[g+1] whose least squared distance to a
 * member is smallest, sorted by (that distance, position).  cand_idx must hold
 * n_grp * n_cand entries.  pts in the renumbered elimination order.  [host] */
sic_status sic_prep_candidates_groups(const double* pts, int64_t n, int32_t dim, const int64_t* grp_ptr,
                                      int64_t n_grp, int32_t n_cand, int64_t* cand_ptr, int32_t* cand_idx,
                                      int32_t n_threads);

/* Candidate lists of nonadjacent groups for partial selection (Section 5.1.1): group g's
 * members are the positions members[grp_ptr[g] .. grp_ptr[g+1]) (ascending, any spacing:
 * e.g. the `members` output of sic_prep_groups, in the original elimination order); its
 * candidates are the n_cand points after its first member, other than its members, whose
 * least squared distance to a member is smallest, sorted by (that distance, position) --
 * so some lie between members and condition only the members before them.  cand_idx must
 * hold n_grp * n_cand entries.  [host] */
sic_status sic_prep_candidates_partial(const double* pts, int64_t n, int32_t dim, const int64_t* members,
                                       const int64_t* grp_ptr, int64_t n_grp, int32_t n_cand, int64_t* cand_ptr,
                                       int32_t* cand_idx, int32_t n_threads);

/* Slices of one factor for several GPUs (Section 4: units are independent; see "one factor
 * built in slices" below): contiguous unit ranges, part r = units bounds[r] .. bounds[r+1]-1
 * (bounds[n_parts + 1], bounds[0] = 0, bounds[n_parts] = n_units), cut where the running
 * estimated cost crosses r / n_parts of the total, so every part's cost is within one
 * unit's cost of the even share.  Cost of unit u with C_u = min(cand_ptr[u+1] - cand_ptr[u],
 * max_cand) candidates and m_u targets (grp_ptr[u+1] - grp_ptr[u]; 1 when grp_ptr is NULL),
 * n_u = k + m_u:  C_u (k^2 + k m_u + m_u^2 / 2) + 13 (n_u^3 / 6 + m_u n_u^2 / 2)  -- the
 * selection's FP32 multiply-adds (two partial factors, k picks) plus the fill's FP64
 * multiply-adds, weighted by 13, the measured ratio of the fill's time per FP64
 * multiply-add to the selection's time per FP32 multiply-add on GB300.  max_cand: the
 * candidates the selection will see (e.g. the proposal's top count), <= 0 for all.  [host] */
sic_status sic_prep_partition(const int64_t* cand_ptr, const int64_t* grp_ptr, int64_t n_units, int32_t k,
                              int32_t max_cand, int32_t n_parts, int64_t* bounds);

/* Candidates for directed GP regression (Section 3): pts holds the n_targets target
 * points first, then the training points.  For each target i < n_targets, the n_cand
 * training positions (>= n_targets) nearest to it, sorted by (distance, position), go
 * to cand_idx[cand_ptr[i] .. cand_ptr[i+1]) (fewer if there are fewer training points).
 * cand_ptr[n_targets + 1], cand_idx[n_targets * n_cand].  [host] */
sic_status sic_prep_candidates_targets(const double* pts, int64_t n, int32_t dim, int64_t n_targets,
                                       int32_t n_cand, int64_t* cand_ptr, int32_t* cand_idx, int32_t n_threads);

/* ---------------------------------------------------------- selection [device] -- */

/* Directed GP selection (Section 3): pick up to k of the n training points x_train
 * [device, n x dim] for the single target x_target [device, dim] by greedy
 * conditional variance reduction.  out_idx[k] [device] receives training indices in
 * pick order (-1 padding), out_var[k+1] [device] the target's conditional variance
 * after t picks (t = 0..count; unused tail untouched), *out_count [device] the number
 * of picks (fewer than k if candidates run out or are exhausted).  Needs
 * sic_select_single_workspace bytes of ws. */
sic_status sic_select_single_workspace(int64_t n, int32_t k, sic_precision prec, size_t* bytes);
sic_status sic_select_single(sic_handle* h, const double* x_train, int64_t n, const double* x_target,
                             const sic_kernel* kp, int32_t k, sic_precision prec, int32_t* out_idx,
                             double* out_var, int32_t* out_count, void* ws, size_t ws_bytes, void* stream);

/* Per-column selection of the factor's sparsity (Section 4).  Column c targets
 * position targets[c] (or c when targets is NULL); its candidates are
 * cand_idx[cand_ptr[c] .. cand_ptr[c+1]) (positions after the target, nearest first).
 * sel_idx[n_cols * k] [device] receives the picked positions in pick order (-1
 * padding); sel_count[n_cols] [device] the number of picks.  All columns run in one
 * persistent launch.  Limits: 1 <= k <= 64, every candidate count <= max_cand <= 1024
 * (max_cand is the caller's bound on cand_ptr[c+1]-cand_ptr[c]; a column above it is
 * reported as SIC_ERR_INVALID by sic_sync); k > 32 needs max_cand <= 512 in FP32 and
 * max_cand <= 256 in FP64, k in 17..32 with max_cand > 512 needs FP32 (SIC_ERR_UNSUPPORTED
 * otherwise).  No workspace. */
sic_status sic_select_columns(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                              const int32_t* targets, int64_t n_cols, const int64_t* cand_ptr,
                              const int32_t* cand_idx, int32_t max_cand, int32_t k, sic_precision prec,
                              int32_t* sel_idx, int32_t* sel_count, void* stream);

/* Supernodal selection (Section 5.2): group g is the consecutive positions
 * grp_ptr[g] .. grp_ptr[g+1]-1 (m_g members, 1 <= m_g <= max_m <= 64); its
 * candidates cand_idx[cand_ptr[g] .. cand_ptr[g+1]) all lie after the group
 * (count <= max_cand <= 4096).  Candidates are scored by var_j / var_j|P, the ratio
 * of their conditional variance given the picks to that given the picks and the
 * targets (eq. greedy_mult).  sel_idx[n_grp * k], sel_count[n_grp] [device] as in
 * sic_select_columns.  1 <= k <= 128.  grp_ptr, cand_ptr [device].  The workspace
 * (sic_select_aggregated_workspace bytes, [device]) also holds the launches' work counters,
 * which the call zeroes on the stream itself; one call at a time per workspace. */
sic_status sic_select_aggregated_workspace(sic_handle* h, int64_t n_grp, int32_t max_cand, int32_t max_m,
                                           int32_t k, sic_precision prec, size_t* bytes);
sic_status sic_select_aggregated(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                 const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                 const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                 sic_precision prec, int32_t* sel_idx, int32_t* sel_count, void* ws,
                                 size_t ws_bytes, void* stream);

/* Partial selection for nonadjacent groups (Section 5.2 "Partial selection", Appendix
 * C.3): group g's targets are members[grp_ptr[g] .. grp_ptr[g+1]) (ascending positions,
 * 1 <= m <= max_m <= 64), its candidates cand_idx[cand_ptr[g] .. cand_ptr[g+1]) (count <=
 * max_cand, each after the group's first member); a candidate conditions only the
 * members before it.  Greedy on sum_i log Theta_{ii | s_i \ i} over the members (eq.
 * partial_kl), s_i = later members and picks after i, with the Cholesky factor of the
 * targets and picks (columns latest first) updated by insertion and in-place rank-one
 * downdate.  Ties: the earliest candidate; a candidate is exhausted when its variance
 * given every member and pick is below sic_exhaustion_floor.  sel_idx[n_grp * k],
 * sel_count[n_grp] as in sic_select_aggregated; gain (n_grp * k FP64, may be NULL) the
 * pick's decrease of the objective per nonzero (per member it conditions; Section 5.4.2).
 * The factor lives in shared memory: (max_cand + max_m) * (max_m + k + 1) values plus
 * small arrays must fit in ~223 KB (SIC_ERR_UNSUPPORTED otherwise), e.g. FP32 with
 * 256 candidates and FP64 with 128, at max_m = k = 64.  1 <= k <= 128.  [device] */
sic_status sic_select_partial(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                              const int64_t* grp_ptr, const int64_t* members, int64_t n_grp, const int64_t* cand_ptr,
                              const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                              sic_precision prec, int32_t* sel_idx, int32_t* sel_count, double* gain, void* stream);

/* The pattern of a partial selection as single-column lists: member i of group g gets
 * col_sel[i * kc ..] = the later members of g, then g's picks after i, and col_count[i] their
 * number (kc >= max_m - 1 + k; a longer list is cut and reported as SIC_ERR_INVALID).  With
 * col_sel NULL only col_count is written (the input of sic_factor_nnz with grp_ptr NULL for
 * sic_build_factor_partial).  The lists also suit sic_build_factor with grp_ptr NULL, max_m
 * 1 and k = kc (one factorisation per column).  Columns of positions in no group are not
 * written.  [device] */
sic_status sic_partial_columns(sic_handle* h, int64_t n, const int64_t* grp_ptr, const int64_t* members,
                               int64_t n_grp, const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                               int32_t kc, int32_t* col_sel, int32_t* col_count, void* stream);

/* KL-optimal FP64 fill of a partial-selection pattern, aggregated per group (Section 5.1.1,
 * Appendix A.4): the group's members and picks sorted from the latest position to the
 * earliest make every member's set a leading block, so one LDL^T of Theta over them serves
 * all members (member u_a: L_S^T x = e_a d_a^{-1/2} over the leading block, log v = log
 * d_a).  col_ptr from sic_factor_nnz (grp_ptr NULL) on the counts of sic_partial_columns;
 * row_idx / val / logv / *sum_logv as in sic_build_factor.  Positions of a group's union
 * must be distinct and its picks after its first member (else SIC_ERR_INVALID by
 * sic_sync).  max_m <= 64, k <= 128, (max_m + k) <= 192.  ws: sic_build_factor_workspace(n)
 * bytes.  [device] */
sic_status sic_build_factor_partial(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                    const int64_t* grp_ptr, const int64_t* members, int64_t n_grp, int32_t max_m,
                                    const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                                    const int64_t* col_ptr, int32_t* row_idx, double* val, double* logv,
                                    double* sum_logv, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------- global allocation of nonzeros [device] -- */
/*
 * Section 5.4: instead of k picks everywhere, a budget of off-diagonal nonzeros goes to
 * whichever unit (column or supernode) lowers the KL divergence most per nonzero.  The
 * paper keeps every unit's best candidate in a priority queue; here each unit first runs
 * its local greedy for up to k picks, reporting the exact decrease of each pick, and
 * sic_allocate_global then keeps a prefix of every unit's picks.  The prefixes equal
 * what the queue would pop (a unit's candidates change only when the unit itself gains
 * an entry, so its picks come in its local order; a pick is popped once the running
 * minimum of its unit's decreases up to it is the largest left).
 *
 * sic_select_columns_gain / sic_select_aggregated_gain: as sic_select_columns /
 * sic_select_aggregated, plus gain[n_units * k] [device, FP64]: gain[u * k + t] is the
 * decrease per nonzero of 2 KL by pick t (t < sel_count[u]; later entries untouched):
 *   column (Section 5.4.1, eq. global_obj): log(v_t / v_{t+1}), v_t the target's
 *     conditional variance after t picks, i.e. -log(1 - corr^2) of the pick;
 *   supernode of m members (Section 5.4.2): log(Theta_{jj|I} / Theta_{jj|I,P}) / m for
 *     the pick j (the change of logdet Theta_{PP|I}; the pick adds m nonzeros).
 * In SIC_FP32_MIXED the ratio comes from the FP32 selection state, the logarithm in FP64.
 */
sic_status sic_select_columns_gain(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                   const int32_t* targets, int64_t n_cols, const int64_t* cand_ptr,
                                   const int32_t* cand_idx, int32_t max_cand, int32_t k, sic_precision prec,
                                   int32_t* sel_idx, int32_t* sel_count, double* gain, void* stream);
sic_status sic_select_aggregated_gain(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                      const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                      const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                      sic_precision prec, int32_t* sel_idx, int32_t* sel_count, double* gain,
                                      void* ws, size_t ws_bytes, void* stream);

/* FP64 side state of a selection (the FP32 path's FP64 pivot conditional variances):
 * for the picks q_0, q_1, ... of every unit (sel_idx[u * k .. u * k + sel_count[u]), in
 * pick order, as returned by the selection calls in either precision) it computes in FP64
 *   pvar[u * k + t]   = Theta_{q_t q_t | q_0..q_t-1}        (conditioned on earlier picks),
 *   pvar_p[u * k + t] = Theta_{q_t q_t | P, q_0..q_t-1}     (and on the unit's targets P),
 *   gain[u * k + t]   = log(pvar / pvar_p) / m              (the pick's exact decrease of
 *                                                          logdet Theta_{PP|I} per nonzero,
 *                                                          eq. greedy_mult / eq. global_obj),
 * from LDL^T factorisations of Theta_SS and of Theta over [P; S] (their pivots are these
 * conditional variances; eq. cond_select).  Units: supernodes grp_ptr[u] .. grp_ptr[u+1]-1
 * (1 <= m <= max_m <= 64), or with grp_ptr NULL single columns targeting targets[u] (u
 * when NULL; max_m must be 1).  1 <= k <= 128.  Any of pvar, pvar_p, gain may be NULL (not
 * all); entries from sel_count[u] on are untouched.  A pick outside [0, n) or a unit
 * outside its bounds is reported by sic_sync as SIC_ERR_INVALID, a repeated pick (a
 * singular Theta_SS) as SIC_ERR_NOT_PD; that unit's entries are then NaN.  [device] */
sic_status sic_side_state_fp64(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                               const int64_t* grp_ptr, const int32_t* targets, int64_t n_units, int32_t max_m,
                               const int32_t* sel_idx, const int32_t* sel_count, int32_t k, double* pvar,
                               double* pvar_p, double* gain, void* stream);

/* Global greedy allocation (Section 5.4) of `budget` off-diagonal nonzeros over n_units
 * units with the gains above.  A pick of unit u costs m_u nonzeros (m_u = grp_ptr[u+1] -
 * grp_ptr[u]; 1 for every unit when grp_ptr is NULL).  Picks are taken in the queue's
 * order -- largest running minimum of the unit's gains first, equal keys by lower unit,
 * then earlier pick -- until the first pick whose cost exceeds what is left of the budget.
 * out_count[n_units] [device] receives the number of leading picks kept per unit
 * (<= sel_count[u]); the pattern is sel_idx[u * k .. u * k + out_count[u]), to be passed
 * as sel_count to sic_factor_nnz and sic_build_factor.  gain, sel_count, grp_ptr
 * [device]; budget >= 0; 1 <= k <= 128.  A sel_count outside [0, k] or a NaN gain is
 * reported by sic_sync as SIC_ERR_INVALID (that unit is then treated as empty, or the
 * NaN as -infinity).  Needs sic_allocate_global_workspace bytes of ws. */
sic_status sic_allocate_global_workspace(int64_t n_units, int32_t k, size_t* bytes);
sic_status sic_allocate_global(sic_handle* h, int64_t n_units, const int64_t* grp_ptr, const double* gain,
                               const int32_t* sel_count, int32_t k, int64_t budget, int32_t* out_count, void* ws,
                               size_t ws_bytes, void* stream);

/* ----------------------------------------------------------- the factor [device] -- */

/* Column pointers of the factor for a selection.  Without groups (grp_ptr NULL,
 * n_grp = n) column i holds 1 + sel_count[i] entries; with groups, member a of a
 * group of m holds (m - a) + sel_count[g] entries (itself, the later members, the
 * shared picks; Section 5.1).  col_ptr[n+1] [device].  Needs sic_factor_nnz_workspace
 * bytes of ws.  The total nnz is col_ptr[n]. */
sic_status sic_factor_nnz_workspace(int64_t n, size_t* bytes);
sic_status sic_factor_nnz(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp, const int32_t* sel_count,
                          int64_t n, int64_t* col_ptr, void* ws, size_t ws_bytes, void* stream);

/* Allocation-free variant of sic_factor_nnz (the paper has no counterpart; it is a
 * convenience of this library).  For callers that cannot allocate device memory --
 * for example code running inside a host framework that has reserved the device's
 * memory for its own allocator, or a latency-critical loop where cudaMalloc's implicit
 * device synchronisation is not acceptable -- and so cannot provide the workspace of
 * sic_factor_nnz.  Same arguments and result as sic_factor_nnz without the workspace.
 * Its scratch is a fixed static device array inside libsic (512 KiB, held by every GPU
 * that loads the library until the process exits), so n + 1 may not exceed
 * 67,108,864 (= 2^26); larger n returns SIC_ERR_UNSUPPORTED.  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  Outside stream
 * capture every call looks up the array's device address (cudaGetSymbolAddress) on the
 * current device, so a device reset between calls is harmless; a call made while `stream`
 * is being captured reuses the address of the last uncaptured call on that device, so make
 * one call on the device before any capture (else SIC_ERR_CUDA).  All calls share the one array and it
 * keeps the last call's contents (nothing in it needs to start at zero): calls that
 * may overlap on the GPU -- on different streams without an ordering between them, or
 * from several threads -- race on it and must be serialised by the caller. */
sic_status sic_factor_nnz_noalloc(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp, const int32_t* sel_count,
                                  int64_t n, int64_t* col_ptr, void* stream);

/* KL-optimal fill (eq. L_col; aggregated form of Appendix A.4) in FP64 for the
 * pattern sel_idx / sel_count (k picks per column or group, as returned by the
 * selection calls; any order).  Writes row_idx / val at col_ptr (from
 * sic_factor_nnz), logv[n] = log Theta_{ii | s_i \ i} and *sum_logv (one FP64 on the
 * device, summed in a fixed order so that repeated runs agree bit for bit).  The KL
 * divergence of the factor is (sum_logv - logdet Theta) / 2 (eq. obj_chol).
 * grp_ptr NULL means single columns (n_grp = n).  max_m bounds the group size (1
 * without groups, <= 64).  Needs sic_build_factor_workspace bytes of ws (the fixed-order sum's
 * partials and the launches' work counters, which the call zeroes on the stream itself; one
 * call at a time per workspace). */

sic_status sic_build_factor_workspace(int64_t n, size_t* bytes);
/* Autotuned variant (this library's launch tuning; the paper has no counterpart): the same
 * arguments and results as sic_build_factor, but it runs the fill once per candidate split of
 * the group-size classes (groups of <= split members in the 4-worker launch, larger in the
 * 8-worker one; candidates 8 .. 64 capped at max_m), times each with CUDA events on `stream`
 * (synchronising it; not for stream capture), keeps the fastest in the handle for this
 * (k, max_m), then times 8 against 12 worker warps for the large-group launch at that split;
 * later sic_build_factor calls with the same k and max_m use both choices; it leaves the
 * outputs of the chosen configuration (they do not depend on either choice).  *best_split [host]
 * receives the choice (may be NULL).  sic_tune_save / sic_tune_load write and read the
 * handle's table as text ("op a b value ms" per line, op 1 = the split, op 2 = the
 * large-group launch's worker threads (256 or 384), a = k, b = max_m; op 3 = the supernodal
 * selection's plan of sic_tune_select_aggregated, a = k + 256 prec, b = 128 max_cand + max_m);
 * a line that does not parse is skipped and reported as SIC_ERR_INVALID.  sic_tune_count /
 * sic_tune_entry list the table.  [device / host] */
sic_status sic_tune_build_factor(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                 const int64_t* grp_ptr, int64_t n_grp, int32_t max_m, const int32_t* sel_idx,
                                 const int32_t* sel_count, int32_t k, const int64_t* col_ptr, int32_t* row_idx,
                                 double* val, double* logv, double* sum_logv, void* ws, size_t ws_bytes,
                                 void* stream, int32_t* best_split);
/* Autotuned launch plan of the supernodal selection (this library's launch tuning; the paper
 * has no counterpart): the same arguments and results as sic_select_aggregated, but it runs
 * the selection once per launch plan that gives the same picks -- threads per CTA (128 or 256
 * for the register-resident FP32 kernel with at most 128 candidates; 256 or 512 for the
 * generic kernel) and the generic kernel's state in shared memory (when it fits) or in the
 * workspace (when `ws` holds it) --, each three times with CUDA events on `stream`
 * (synchronising it; not for stream capture), keeps the fastest in the handle for (k, prec,
 * max_cand, max_m) (op 3 of the table: value = 2 * threads + 1 if in shared memory, or the
 * register kernel's threads), and leaves the picks of a final run with it.  Later
 * sic_select_aggregated calls in that bucket use it (the default plan when the given
 * workspace is too small for it).  *choice [host] receives the value (may be NULL).
 * SIC_ERR_INVALID when no plan fits the given workspace.  [device / host] */
sic_status sic_tune_select_aggregated(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                      const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                      const int32_t* cand_idx, int32_t max_cand, int32_t max_m, int32_t k,
                                      sic_precision prec, int32_t* sel_idx, int32_t* sel_count, void* ws,
                                      size_t ws_bytes, void* stream, int32_t* choice);
sic_status sic_tune_save(const sic_handle* h, const char* path);
sic_status sic_tune_load(sic_handle* h, const char* path);
int32_t sic_tune_count(const sic_handle* h);
sic_status sic_tune_entry(const sic_handle* h, int32_t i, int32_t* op, int32_t* a, int32_t* b, int32_t* value,
                          float* ms);
sic_status sic_build_factor(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                            const int64_t* grp_ptr, int64_t n_grp, int32_t max_m, const int32_t* sel_idx,
                            const int32_t* sel_count, int32_t k, const int64_t* col_ptr, int32_t* row_idx,
                            double* val, double* logv, double* sum_logv, void* ws, size_t ws_bytes,
                            void* stream);

/* ------------------------------------------ one factor built in slices [device] -- */
/*
 * Section 4: the columns (or supernodes) of the factor are independent of one another, so
 * one factor can be built in slices -- contiguous ranges of units, e.g. one per GPU, every
 * slice holding all the points -- and the slices' CSC pieces concatenated.  A slice is the
 * units u0 .. u1-1 of the whole problem: grp_ptr + u0 (n_grp = u1 - u0 groups, positions
 * unchanged) or, without groups, the single columns u0 .. u1-1 (selected with
 * sic_select_columns' `targets` = u0 .. u1-1); its columns are col0 .. col0 + n_cols - 1
 * (col0 = grp_ptr[u0] or u0).
 *
 * sic_factor_nnz_range: col_ptr[0 .. n_cols] [device] for the slice's columns, starting at
 * `base` (col_ptr[c - col0] is the offset of column c; base = 0 for a slice's own arrays, or
 * the entries of all earlier slices for the whole factor's col_ptr).  Units outside the
 * column range are reported by sic_sync as SIC_ERR_INVALID.  ws: sic_factor_nnz_workspace(
 * n_cols) bytes.  sic_factor_nnz is the case col0 = 0, n_cols = n, base = 0.
 *
 * sic_build_factor_range: the fill of the slice (pts, n: all points).  Column c's entries go
 * to row_idx / val at col_ptr[c - col0] - base, so row_idx / val hold just the slice's
 * col_ptr[n_cols] - base entries; logv[n_cols] receives log v of the slice's columns and
 * *sum_logv their fixed-order sum.  ws: sic_build_factor_workspace(n_cols) bytes.
 * sic_build_factor is the case col0 = 0, n_cols = n, base = 0; the entries of a column do
 * not depend on the slicing (each unit's arithmetic is the same).
 *
 * sic_sum_fixed: *sum [device] = the sum of x[0 .. n) [device] in the fixed order of
 * sic_build_factor's sum_logv (tiles of 2048, then the tile sums), so that the log v of a
 * factor gathered from slices sums to the bit-identical value of one whole build.  ws:
 * sic_build_factor_workspace(n) bytes. */
sic_status sic_factor_nnz_range(sic_handle* h, const int64_t* grp_ptr, int64_t n_grp, const int32_t* sel_count,
                                int64_t col0, int64_t n_cols, int64_t base, int64_t* col_ptr, void* ws,
                                size_t ws_bytes, void* stream);
sic_status sic_build_factor_range(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                  const int64_t* grp_ptr, int64_t n_grp, int32_t max_m, const int32_t* sel_idx,
                                  const int32_t* sel_count, int32_t k, int64_t col0, int64_t n_cols,
                                  const int64_t* col_ptr, int64_t base, int32_t* row_idx, double* val, double* logv,
                                  double* sum_logv, void* ws, size_t ws_bytes, void* stream);
sic_status sic_sum_fixed(sic_handle* h, const double* x, int64_t n, double* sum, void* ws, size_t ws_bytes,
                         void* stream);

/* y = op(L) x for the CSC factor; x, y are n x nrhs row-major FP64 (x[r * nrhs + c]),
 * 1 <= nrhs <= 8, all [device].  SIC_OP_L: y = L x; SIC_OP_LT: y = L^T x;
 * SIC_OP_LLT: y = L (L^T x), the preconditioner (L L^T ~ Theta^{-1}).  x and y must
 * not overlap.  Needs sic_apply_factor_workspace bytes of ws (the intermediate of
 * SIC_OP_LLT). */
sic_status sic_apply_factor_workspace(int64_t n, int32_t nrhs, sic_op op, size_t* bytes);
sic_status sic_apply_factor(sic_handle* h, int64_t n, const int64_t* col_ptr, const int32_t* row_idx,
                            const double* val, sic_op op, const double* x, double* y, int32_t nrhs, void* ws,
                            size_t ws_bytes, void* stream);

/* ------------------------------------------------- preconditioning [device] -- */

/* y = (Theta + shift I) x without forming Theta (O(n^2) kernel evaluations), x, y
 * n x nrhs row-major FP64, 1 <= nrhs <= 8.  SIC_FP32_MIXED evaluates the kernel entries
 * in FP32 (a fixed symmetric rounding of Theta) and sums the products with double-FP32
 * compensated arithmetic (x split into two FP32 parts), tiles added in FP64; SIC_FP64
 * is FP64 throughout (reference for small n).  x and y must not overlap. */
sic_status sic_matern_matvec(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp, double shift,
                             sic_precision prec, const double* x, double* y, int32_t nrhs, void* stream);

/* Preconditioned conjugate gradients for (Theta + shift I) x = b, nrhs <= 8 right-hand
 * sides solved together (the use of the factor as a preconditioner, Section 6.4):
 * M^{-1} = L L^T from the CSC factor (col_ptr, row_idx, val), or no preconditioner when
 * all three are NULL.  Starts from x = 0; a right-hand side stops when its recursively
 * updated residual satisfies |r| / |b| < tol or after max_iter iterations.  iters[nrhs]
 * and relres[nrhs] are HOST arrays receiving the iteration counts and final relative
 * residuals.  The call synchronises the stream once per iteration (the loop runs on the
 * host).  ws: sic_pcg_workspace bytes. */
sic_status sic_pcg_workspace(int64_t n, int32_t nrhs, size_t* bytes);
sic_status sic_pcg_solve(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp, double shift,
                         sic_precision prec, const int64_t* col_ptr, const int32_t* row_idx, const double* val,
                         const double* b, double* x, int32_t nrhs, double tol, int32_t max_iter, int32_t* iters,
                         double* relres, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------ learned proposal [device] -- */
/*
 * Not part of the paper: a small MLP ranks each supernode's candidates so that the
 * exact greedy selection above runs only on the `top` best of them; the plain greedy
 * stays the reference (and the source of the training labels).
 *
 * Features: 8 FP32 per candidate, row-major feat[(cand_ptr[g] + r) * 8 + f], for the
 * group P = grp_ptr[g] .. grp_ptr[g+1]-1 (m <= 64 members) with R the distance from
 * the group's last (farthest) candidate to its nearest member (1 if zero), a* the
 * nearest member (lowest index on ties), K the kernel without nugget:
 * f0, f1 = (x_j - x_a*)[0], [1] / R;  f2 = |x_j - x_a*| / R;  f3 = |x_j - centroid(P)| / R;
 * f4 = r / C;  f5 = K(|x_j - x_a*|) / variance;  f6 = m / 64;
 * f7 = mean over members of K(|x_j - x_a|) / variance.  Computed in FP32 from
 * coordinates taken relative to the group's first member in FP64.
 *
 * Network: s = w3 . gelu(W2^T gelu(W1^T f + b1) + b2) + b3 with exact (erf) GELU,
 * 8 -> 128 -> 128 -> 1.  Parameters are one flat FP32 array of sic_mlp_param_count()
 * = 17793 values: W1 [8][128] (row = input), b1 [128], W2 [128][128] (row = input),
 * b2 [128], w3 [128], b3 [1].
 */
int32_t sic_mlp_param_count(void);

/* feat must hold cand_ptr[n_grp] * 8 floats [device], 16-byte aligned (each candidate's row is
 * written as two 16-byte words); a misaligned feat returns SIC_ERR_INVALID. */
sic_status sic_proposal_features(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp,
                                 const int64_t* grp_ptr, int64_t n_grp, const int64_t* cand_ptr,
                                 const int32_t* cand_idx, float* feat, void* stream);

/* score[rows] = the network applied to feat[rows x 8] on the tcgen05 tensor cores: BF16
 * weights and inputs, FP32 accumulation in tensor memory, the hidden activations rounded
 * to BF16 as the second layer's input.  No workspace. */
sic_status sic_proposal_score(sic_handle* h, const float* params, const float* feat, int64_t rows, float* score,
                              void* stream);

/* Keeps, per group, the min(top, C) candidates of highest score (ties: earlier in the
 * list), in their original list order.  out_ptr[n_grp+1] receives the CSR offsets,
 * out_idx must hold n_grp * top entries.  C <= 4096. */
sic_status sic_proposal_topk(sic_handle* h, const int64_t* cand_ptr, const int32_t* cand_idx, const float* score,
                             int64_t n_grp, int32_t top, int64_t* out_ptr, int32_t* out_idx, void* stream);

/* label[cand_ptr[g] + r] = 1 if candidate r of group g is among the picks sel_idx[g*k ..
 * g*k + sel_count[g]) of a selection (the training labels), else 0.  k <= 256. */
sic_status sic_proposal_labels(sic_handle* h, const int64_t* cand_ptr, const int32_t* cand_idx, int64_t n_grp,
                               const int32_t* sel_idx, const int32_t* sel_count, int32_t k, float* label,
                               void* stream);

/* Training (FP32): loss = mean over the batch of
 * pos_weight * y * softplus(-s) + (1 - y) * softplus(s), and its gradient with respect
 * to the flat parameters (grads, same layout).  With bf16 != 0 the forward pass uses
 * BF16-rounded weights, inputs and first-layer activations, as inference does (the
 * gradient passes straight through the rounding).  score[batch] (optional, may be NULL)
 * receives the logits, *loss the mean loss [device].  ws: sic_mlp_train_workspace. */
sic_status sic_mlp_train_workspace(int64_t batch, size_t* bytes);
sic_status sic_mlp_grads(sic_handle* h, const float* params, const float* feat, const float* label, int64_t batch,
                         float pos_weight, int32_t bf16, float* grads, float* loss, float* score, void* ws,
                         size_t ws_bytes, void* stream);

/* One AdamW step (decoupled weight decay, bias-corrected moments; step counts from 1)
 * on n parameters: m, v are the moment buffers [device]. */
sic_status sic_adamw_step(sic_handle* h, float* params, float* m, float* v, const float* grads, int32_t n,
                          int32_t step, float lr, float beta1, float beta2, float eps, float wd, void* stream);

/* ------------------------------------------------- directed GP regression -- */

/* Posterior of the latent process at targets[t] (positions of pts) given the
 * observations y at its picks sel_idx[t * k .. t * k + sel_count[t]) (Section 3, the
 * prediction step after the directed selection; e.g. picks from sic_select_columns on
 * candidates from sic_prep_candidates_targets):
 *   mean[t] = Theta_{t,I} Theta_{I,I}^{-1} y_I,
 *   var[t]  = variance - Theta_{t,I} Theta_{I,I}^{-1} Theta_{I,t}
 * in FP64; the nugget (observation noise) sits on the diagonal of Theta_{I,I} only.
 * pts [device, n x dim], targets [device, n_targets] (NULL: t), sel_idx, sel_count
 * [device], y [device, n; only picked positions are read], mean, var [device,
 * n_targets].  1 <= k <= 128.  A pick outside [0, n) or equal to the target, or a
 * count outside [0, k], records SIC_ERR_INVALID; a non-positive pivot (repeated picks)
 * SIC_ERR_NOT_PD (the target's outputs are NaN).  No workspace. */
sic_status sic_gp_predict(sic_handle* h, const double* pts, int64_t n, const sic_kernel* kp, const int32_t* targets,
                          int64_t n_targets, const int32_t* sel_idx, const int32_t* sel_count, int32_t k,
                          const double* y, double* mean, double* var, void* stream);

/* ------------------------------------------------------------ self-test -- */

/* Exercises the bounded device wait used by the tensor-core kernels (not part of the
 * paper): one CTA waits on an mbarrier that nothing arrives at, for at most `cap`
 * polls (1 <= cap <= 2^24), then writes 0 to out[0] [device] and records
 * SIC_ERR_TIMEOUT (unit -2) for sic_sync -- the path a kernel takes when an awaited
 * tensor-core operation never completes; the context stays usable. */
sic_status sic_selftest_wait_timeout(sic_handle* h, int64_t cap, int32_t* out, void* stream);

/* Evaluates the FP64 device routines behind the fill (not part of the paper) on n inputs
 * x[i] >= 0 [device]: out_sqrt[i] = sqrt(x[i]) and out_rsqrt[i] = 1/sqrt(x[i]) by the
 * Newton-refined routines (out_rsqrt undefined at x = 0), out_exp[i] = exp(-x[i]) by the
 * table-driven exponential, and out_kernel[i] = the Matern covariance of *kp (no nugget)
 * at squared distance x[i], all [device, n doubles].  Tests compare them with the
 * library and oracle functions. */
sic_status sic_selftest_fp64_math(sic_handle* h, const sic_kernel* kp, const double* x, int64_t n,
                                  double* out_sqrt, double* out_rsqrt, double* out_exp, double* out_kernel,
                                  void* stream);

/* The fill's integer arithmetic on independent inputs (not part of the paper), for tests:
 * d2[i] = the squared distance between points pa[i] and pb[i] (n x dim, dim 1..3) from their
 * fixed-point coordinates (each dimension at the larger of the two points' exponents; exact
 * differences and squares, one rounding), dot[i] = sum_j ga[i][j] gb[i][j] of two 4-vectors
 * (n x 4) in the panels' fixed-point form (53-bit significands at each vector's largest
 * exponent, exact 32 x 32-bit products, the sum truncated below 2^-51 of the largest product).
 * All pointers [device]; d2, dot: n doubles each. */
sic_status sic_selftest_fixed_point(sic_handle* h, const double* pa, const double* pb, int64_t n, int32_t dim,
                                    double* d2, const double* ga, const double* gb, double* dot, void* stream);

/* Evaluates the double-float Matern of the fill (not part of the paper): out[i] = the kernel
 * of *kp (no nugget) between points pa[i] and pb[i] (n x dim each, [device]), computed as the
 * fill computes its entries -- coordinates relative to an origin (here pa[i]) split into
 * double-floats, distance, square root and table-driven exponential in double-float
 * arithmetic on the FP32 pipe, one FP64 addition at the end.  out [device, n doubles].  Tests
 * compare it with the FP64 oracle (absolute error a few 1e-15 of the variance). */
sic_status sic_selftest_matern_df(sic_handle* h, const sic_kernel* kp, const double* pa, const double* pb, int64_t n,
                                  double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SIC_H */
