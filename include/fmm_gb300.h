/*
 * fmm_gb300.h -- C ABI of the GB300 (sm_103a) periodic fast multipole method
 * for a net-charged cubic box neutralised by a uniform background charge
 * (Urano, Shinoda, Yoshii & Okazaki, arXiv:2003.13218).
 *
 * Problem statement (Appendix A): N point charges q_i at r_i in a cubic unit
 * cell of side b (volume V = b^3) under periodic boundary conditions, plus a
 * uniform background charge of density -Q_C / V (Q_C = sum q_i), with the
 * conducting boundary at infinity.  The energy evaluated is Eq. Velecfull:
 *
 *   V_elec = 1/2 sum_i q_i sum_{j in NF(i)} q_j / r_ij            (Eq. EqNF)
 *          + 1/2 sum_i q_i sum_{n,m} L_n^m(l_max) R_n^m(r_i - r_L') (Eq. EqFF)
 *          - pi Q_C^2 / (2 V kappa^2)                               (Eq. 6)
 *          + (2 pi / 3V) Q_C sum_i q_i r_i^2                       (Eq. surfchargedend)
 *          - (2 pi / 3V) mu . mu                                    (Appendix D)
 *
 * where the local coefficients L come from P2M (Eq. P2M), M2M, the level-0
 * lattice sum over image cells (Eq. 12, with the self term 12c), M2L over each
 * level's interaction list (Eq. Lcoeffdef) and L2L (Appendix B).
 *
 * Units: lengths in A, charges in e, energies in e^2/A (Gaussian units
 * without 1/(4 pi eps0), Appendix A).  Multiply by 1389.35458 for kJ/mol.
 *
 * Conventions shared by every call
 *  - All functions return fmm_status; nothing aborts, traps or exits.
 *  - Position arrays are double[N][3] (x, y, z interleaved), charge arrays
 *    double[N], membership arrays uint8_t[N] (1 = solute).  Pointers may be
 *    device pointers (the fast path) or host pointers; host inputs are copied
 *    to plan-owned device buffers inside the call and host outputs copied back.
 *  - The caller owns every input and output buffer; the plan owns its scratch
 *    memory, operator tables and stream binding.
 *  - Work is enqueued on the plan's stream (default: the legacy default stream;
 *    see FMM_OPT_STREAM).  Calls that return host scalars synchronise that
 *    stream before returning.  With FMM_OPT_OVERLAP (default on) a call forks
 *    from that stream onto plan-owned streams and joins back into it before it
 *    returns: work enqueued on the plan's stream afterwards sees its results.
 *  - A plan is not thread-safe: use one plan per host thread or stream.
 *  - Positions may lie outside [0, b); each atom is wrapped into the cell.
 *  - Non-finite positions or charges yield FMM_ERR_NONFINITE (detected on the
 *    device, reported after the call's kernels have finished).
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s *fmm_plan;

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = 1, /* bad size, order, depth, pointer or option */
    FMM_ERR_NONFINITE = 2,   /* NaN/Inf in positions or charges */
    FMM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    FMM_ERR_OOM = 4,         /* device or host allocation failed */
    FMM_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
    FMM_ERR_INTERNAL = 6,    /* a device-side consistency check failed */
    FMM_ERR_UNSUPPORTED = 7  /* option value not built (e.g. ws > 2) */
} fmm_status;

/* Energy decomposition of Eq. Velecfull, e^2/A. */
typedef struct {
    double near;           /* first term: near-field pair sum (Eq. EqNF) */
    double far;            /* second term: far field via local expansions (Eq. EqFF) */
    double charged;        /* -pi Q_C^2 / (2 V kappa^2) (Eq. 6) */
    double quad_surface;   /* +(2 pi / 3V) Q_C sum q_i r_i^2 (Eq. surfchargedend) */
    double dipole_surface; /* -(2 pi / 3V) mu . mu (Appendix D) */
    double total;          /* compensated sum of the five terms */
} fmm_energy_terms;

/* Parts of the reduced-far-field solute-solvent energy (Eq. FMMcalc). */
typedef struct {
    double e_uv;     /* NF_uv + W + bc_cross: interaction of (solute + its background)
                        with (solvent + its background) */
    double W;        /* far-field interaction, (A - B + C) / 2 */
    double A;        /* sum_{i in u} q_i Phi_{u,v}^FF(r_i)  (full pass) */
    double B;        /* sum_{i in u} q_i Phi_u^FF(r_i)      (solute-only pass) */
    double C;        /* sum_{j in v} q_j Phi_u^FF(r_j)      (solute-only pass) */
    double nf_uv;    /* near-field solute-solvent pair sum */
    double bc_cross; /* -pi Q_u Q_v/(V kappa^2) + (2 pi/3V)(Q_u S2_v + Q_v S2_u)
                        - (4 pi/3V) mu_u . mu_v */
    double nf_sc;    /* FMM_OPT_SOFTCORE: sum over the near-field solute-solvent pairs of
                        q_i q_j / (alpha lambda A^c + r_ij^c)^(1/c) (0 when off) */
    double dnf_sc;   /* its derivative in lambda, -(alpha A^c / c) sum q_i q_j (alpha lambda A^c + r^c)^(-1/c-1) */
} fmm_uv_terms;

/* Per-stage device times of the last call, milliseconds (CUDA events on the
 * stream that runs the far field).  m2l_l2l covers M2L and L2L of levels
 * 1..l_max of the full pass; m2l_kernels the M2L launches alone; solute_pass
 * the part of the solute-only pass of Eq. FMMcalc that runs after the full
 * pass (its prologue overlaps the full pass on a side stream; 0 when not
 * requested); m2l_top the single tensor-core M2L launch of level l_max (0 when
 * that level runs on CUDA cores).  With FMM_OPT_OVERLAP the near field and the
 * sparse solute pass run beside the far field: p2p is then about 0 and
 * solute_pass holds the wait for both and the last solute kernel. */
typedef struct {
    float sort, upward, lattice, m2l_l2l, l2p, p2p, solute_pass, reduce, total, m2l_kernels, m2l_top;
} fmm_timings;

/* Options for fmm_plan_set_option. */
enum {
    FMM_OPT_WS = 1,        /* well-separatedness ws of App. B: 1 (default; 189-cell interaction lists,
                              27-leaf near field) or 2 (the paper's setting: 875 and 125; needs 2^depth > 5);
                              other values FMM_ERR_UNSUPPORTED (> 2) or FMM_ERR_INVALID_ARG */
    FMM_OPT_PRECISION = 2, /* ival: FMM_PREC_FP64 (default) or FMM_PREC_MIXED */
    FMM_OPT_KAPPA = 3,     /* dval: splitting parameter kappa of Eq. 12 and Eq. 6 in 1/A;
                              <= 0 restores the default kappa = 2 / b */
    FMM_OPT_M2L_SPLIT = 4, /* ival: mixed-precision M2L operand split, FMM_SPLIT_* (default FP16X2) */
    FMM_OPT_STREAM = 5,    /* ival: cudaStream_t cast to int64 (0 = legacy default stream) */
    FMM_OPT_TIMINGS = 6,   /* ival: 1 records per-stage CUDA events (adds event overhead) */
    FMM_OPT_M2L_PAIR = 7,  /* ival: 1 (default) lets the fp16x2 tensor-core M2L of levels with an even
                              number of 128-cell tiles per class run on CTA pairs (2-SM MMAs, half the
                              operator traffic per SM); 0 keeps every level on single-CTA MMAs */
    FMM_OPT_BOUNDARY = 8   /* ival: FMM_BOUNDARY_CONDUCTING (default; Eq. Velecfull, with the dipole surface
                              term -(2 pi/3V) mu.mu of App. D) or FMM_BOUNDARY_VACUUM (App. D: FMM's own
                              boundary, without that term, its force and its solute-solvent cross term
                              -(4 pi/3V) mu_u.mu_v) */,
    FMM_OPT_OVERLAP = 9    /* ival: 1 (default) runs a call on plan-owned streams: the far field on one above
                              the default priority, the near field (P2P, which needs only the sort) on one
                              of the lowest priority filling the SMs the far field leaves idle, the sparse
                              solute pass of Eq. FMMcalc beside the L2P; 0 runs every stage in order on the
                              plan's stream (the per-stage times then add up) */,
    FMM_OPT_M2L_GRADE = 10 /* ival = D2 | (D1 << 8), fp16x2 tensor-core M2L only: per K chunk of input coefficients
                              (64 per chunk), by the chunk's lowest degree lambda: lambda >= D1 keeps one product
                              (both operands' first fp16 terms, ~2^-11 relative on those terms) and two
                              consecutive 1-product chunks share one pipeline stage; otherwise each K16 step of
                              the chunk whose lowest degree reaches D2 drops the moments' second fp16 term (2
                              products: ~2^-12 relative on those terms), the other steps keep all 3; 0 = never.  Contributions of high input
                              degrees to a well-separated cell's local expansion are small, so the error stays far
                              below the first-term precision of the low degrees.  D2, D1 in 0..20; default
                              FMM_GRADE_DEFAULT.  M2M, the fused L2L and the solute-only pass always use 3
                              products */,
    FMM_OPT_M2L_ACC_GROUP = 11 /* ival in 1..64: tensor-core M2L / M2M offsets whose products are summed in
                              one FP32 TMEM accumulator before it is drained into registers (the fused L2L
                              always alone); longer chains drain less often but carry more of the tensor
                              core's accumulation rounding; default FMM_ACC_GROUP_DEFAULT */,
    FMM_OPT_SOFTCORE = 12,  /* ival = c (1..12; 0 = off, the default), dval = A (A, > 0): the soft-core form the
                              paper gives for the solute-solvent LJ term (Calculation detail), which it notes
                              applies to the electrostatic NF term too, r_ij -> (alpha lambda A^c + r_ij^c)^(1/c)
                              on the near-field solute-solvent pairs: evaluations that return fmm_uv_terms also
                              return that pair sum and its lambda derivative (nf_sc, dnf_sc; FP64 arithmetic).
                              The paper uses alpha = 0.2 and c = 6 for its LJ lengths A_ij; A is the caller's */
    FMM_OPT_SOFTCORE_LAMBDA = 13, /* dval in [0, 1]: the lambda of that sum (default 0); read when the call runs,
                              so a recorded batch graph sees the current value */
    FMM_OPT_SOFTCORE_ALPHA = 14,  /* dval > 0: alpha (default 0.2) */
    FMM_OPT_WAIT_BUDGET_NS = 15,  /* ival in 1000..10^10: budget (ns) of each bounded wait in the tensor-core
                              kernels (default 2 s); a wait that runs out makes the call return FMM_ERR_TIMEOUT
                              after the kernel has waited, with its own 2 s limit, for its copies and MMAs in
                              flight; the plan stays usable */
    FMM_OPT_INJECT_STALL = 16,    /* ival 0 / 1, a test hook for the timeout path: with 1 the single-CTA
                              tensor-core kernels first wait on a barrier that nothing arrives on, so every
                              evaluation returns FMM_ERR_TIMEOUT after the wait budget (use with
                              FMM_OPT_M2L_PAIR = 0 and a short budget) */
    FMM_OPT_M2L_BRICK = 17        /* ival = l | bx << 8 | by << 16 | bz << 24: the tiles of the tensor-core M2L of
                              level l (2..depth; and the M2M from it) are bricks of bx x by x bz cells of one
                              parity class, bx by bz = 128, each dividing 2^(l-1), an even number per class.
                              Only the grouping of targets into tiles changes: results are bitwise the same.
                              FMM_ERR_UNSUPPORTED without the tensor-core path (FP64 plans); a WS, PRECISION
                              or M2L_SPLIT change restores the default bricks */
};
#define FMM_GRADE_DEFAULT (4 | (8 << 8))  /* D2 = 4, D1 = 8: degrees 4..7 with two products, >= 8 with one */
#define FMM_ACC_GROUP_DEFAULT 2
enum { FMM_BOUNDARY_CONDUCTING = 0, FMM_BOUNDARY_VACUUM = 1 };
enum { FMM_PREC_FP64 = 0, FMM_PREC_MIXED = 1 };
enum {
    FMM_SPLIT_BF16X3 = 0,    /* tensor-core M2L: both operands as 3 bf16 terms, 6 products */
    FMM_SPLIT_BF16X2 = 1,    /* tensor-core M2L: 2 bf16 terms, 3 products */
    FMM_SPLIT_FP32 = 2,      /* FP32 CUDA-core M2L (no tensor cores) */
    FMM_SPLIT_BF16_A2B3 = 3, /* tensor-core M2L: moments in 2 bf16 terms, operators in 3, 4 products */
    FMM_SPLIT_FP16X2 = 4     /* tensor-core M2L: both operands balanced by sqrt((n+m)!(n-m)!) and a power of
                                two, then split into 2 fp16 terms, 3 products (~2^-22 relative) */
};

/*
 * Create a plan for N charges in a cubic box of side `box` (A), with 2^depth
 * leaf cells per side (depth = l_max of Appendix B) and expansion order
 * p = n_max (0 <= n <= n_max, Eq. P2M).
 * Errors: FMM_ERR_INVALID_ARG if box <= 0 or not finite, N < 1, p < 0 or
 * p > 20, depth < 2 or depth > 8 (2^depth must exceed 2 ws + 1 so that the
 * near field never holds a charge's own image); FMM_ERR_OOM; FMM_ERR_CUDA.
 * On success *out owns device memory until fmm_plan_destroy.
 */
fmm_status fmm_plan_create(double box, int64_t N, int depth, int p, fmm_plan *out);

/* Set an option (see FMM_OPT_*).  Changing WS, PRECISION, KAPPA or M2L_SPLIT
 * rebuilds the plan's tables.  FMM_ERR_INVALID_ARG for unknown keys or bad
 * values, FMM_ERR_UNSUPPORTED for values this library does not provide. */
fmm_status fmm_plan_set_option(fmm_plan plan, int key, int64_t ival, double dval);

/*
 * Total energy (Eq. Velecfull).  pos: [N][3], q: [N] (device or host).
 * energy: host out (required).  terms: host out, nullable.
 * Synchronises the plan's stream.
 */
fmm_status fmm_energy(fmm_plan plan, const double *pos, const double *q, double *energy,
                      fmm_energy_terms *terms);

/*
 * Energy and forces F_i = -dV_elec/dr_i: pair forces of the near field, minus
 * q_i times the gradient of the far-field potential (L2P gradient; the FMM
 * bilinear form is symmetric, so this is the exact gradient of Eq. EqFF), and
 * -(4 pi / 3V) q_i (Q_C r_i - mu) from the two surface terms.  The charged
 * term exerts no force.  The energy is piecewise smooth: it is not
 * differentiable where a charge crosses a leaf face.
 * forces: [N][3] out, same memory kind as pos.  energy: host out, nullable
 * (non-null synchronises).
 */
fmm_status fmm_forces(fmm_plan plan, const double *pos, const double *q, double *forces, double *energy);

/*
 * Potentials phi_i = dV_elec/dq_i (V_elec of Eq. Velecfull is a quadratic form
 * in the charges, so sum_i q_i phi_i = 2 V_elec): the near-field pair potential
 * of Eq. EqNF plus the far-field potential of Eq. EqFF (L2P; it includes the
 * charge's own periodic images), plus the derivatives of the background terms,
 * -pi Q_C/(V kappa^2) + (2 pi/3V)(S_2 + Q_C |r_i|^2) - (4 pi/3V) mu.r_i (the
 * last one under the conducting boundary only), r_i the wrapped position.
 * potentials: [N] out, same memory kind as pos.  forces: [N][3] out, nullable
 * (the same evaluation).  energy: host out, nullable (non-null synchronises).
 */
fmm_status fmm_potentials(fmm_plan plan, const double *pos, const double *q, double *potentials, double *forces,
                          double *energy);

/*
 * Solute-solvent interaction energy with the reduced far field (Eq. FMMcalc):
 * one full pass gives A; one pass over the solute charges alone gives B and C.
 * is_solute: uint8 [N] (nonzero = solute).  e_uv: host out (required);
 * terms: host out, nullable.  Synchronises.
 */
fmm_status fmm_solute_solvent_energy(fmm_plan plan, const double *pos, const double *q,
                                     const uint8_t *is_solute, double *e_uv, fmm_uv_terms *terms);

/*
 * One call doing all of the above: energy terms, optional forces (nullable) and
 * optional solute-solvent parts (is_solute and uv both non-null), sharing the
 * full pass between them.  terms and uv are host outputs (nullable); forces has
 * the memory kind of pos.  Synchronises when terms or uv is non-null.
 */
fmm_status fmm_evaluate(fmm_plan plan, const double *pos, const double *q, const uint8_t *is_solute,
                        double *forces, fmm_energy_terms *terms, fmm_uv_terms *uv);

/* Per-stage times of the last call (requires FMM_OPT_TIMINGS = 1). */
fmm_status fmm_plan_get_timings(fmm_plan plan, fmm_timings *out);

/* Number of kernel launches enqueued by the last call. */
int64_t fmm_plan_last_launch_count(fmm_plan plan);

/* Which M2L implementation the plan runs at `level` (1..depth):
 * 0 = FP64 CUDA cores, 1 = FP32 CUDA cores, 2 = tcgen05 tensor cores;
 * -1 for a NULL plan or a level out of range. */
int fmm_plan_m2l_backend(fmm_plan plan, int level);

/* Release the plan and its device memory.  Accepts NULL. */
void fmm_plan_destroy(fmm_plan plan);

/*
 * Batches of independent boxes (lambda windows or trajectory frames of uneven
 * size), for the coupling scheme of Eq. Vswucheme: the Coulomb interaction
 * between solute and solvent (charges and backgrounds) is scaled by
 * (1 - lambda_C), so by Eq. FMMVTI the energy is linear in lambda_C:
 *     V_lambda = E_total - lambda_C E_uv,   dV_lambda/dlambda_C = -E_uv,
 * with E_total of Eq. Velecfull and E_uv the solute-solvent interaction of
 * Eq. FMMcalc plus the background cross terms (as fmm_solute_solvent_energy).
 */
typedef struct fmm_batch_s *fmm_batch;

/*
 * Plans for nbox boxes: box[i] the cell side (A), N[i] the charges, depth[i]
 * and p[i] as in fmm_plan_create.  depth == NULL or depth[i] <= 0: the depth is
 * chosen by timing (for each group of boxes with the same starting guess
 * round(log8(N / 3.8)), the box of median size is timed at the guess and one
 * level either side on uniform test charges).  p == NULL or p[i] < 0: 12.
 * precision: FMM_PREC_MIXED or FMM_PREC_FP64.  Work runs on up to 16 streams
 * the batch owns.  Errors as fmm_plan_create (FMM_ERR_INVALID_ARG for any bad
 * box, N, depth or p); on error nothing is left allocated.
 */
fmm_status fmm_batch_create(int nbox, const double *box, const int64_t *N, const int *depth, const int *p,
                            int precision, fmm_batch *out);

/*
 * What the batch tuner chooses beyond the depth (fmm_batch_create_tuned).
 *   energy_rel_tol  > 0: boxes with p[i] < 0 take the smallest order in {6, 8, 10, 12} whose mixed-precision
 *                   total energy (Eq. Velecfull) stays within this relative error of an FP64 order-15
 *                   evaluation on a water-like test box of every depth group (the depths are tuned first,
 *                   at p = 12): the group's smallest size (fewest charges per leaf, the largest truncation
 *                   error) and its cell: a +2 e ion at the centre (where the cells of every level meet)
 *                   and floor((N - 1) / 3) rigid 3-site waters (O -0.834
 *                   e, H +0.417 e, O-H 0.9572 A, H-O-H 104.52 deg) on a jittered cubic lattice in random
 *                   orientations, at the group's depth.  12 when none does; 0: they take 12.  The budget
 *                   bounds the change against order 15, not the error against the exact energy: at ws = 1
 *                   the expansion converges slowly, and on sparse leaves order 15 itself can differ from the
 *                   Ewald energy by a few 1e-6.
 *   sweep           -1: the persistent sweep (FMM_BATCH_OPT_SWEEP) on or off, whichever replays the recorded
 *                   graph of the whole batch faster on uniform test charges; 0: off; 1: on.
 *   tiles           1: for every depth group with a tensor-core pair level, the tile brick of its deepest
 *                   level (FMM_OPT_M2L_BRICK) is the fastest of the power-of-two bricks bx >= by >= bz of 128
 *                   cells, timed on the group's median box with uniform test charges; 0: the default brick.
 */
typedef struct {
    double energy_rel_tol;
    int sweep;
    int tiles;
} fmm_tune_policy;

/* fmm_batch_create with a tuning policy (fmm_batch_create is this with {0, 1, 0}).  Errors as fmm_batch_create,
 * plus FMM_ERR_INVALID_ARG for a NULL policy, a negative or NaN tolerance or sweep outside -1..1. */
fmm_status fmm_batch_create_tuned(int nbox, const double *box, const int64_t *N, const int *depth, const int *p,
                                  int precision, const fmm_tune_policy *policy, fmm_batch *out);

/* What the tuner measured (each nullable): p_err double[4], the largest relative energy error over the depth
 * groups' test boxes of p = 6, 8, 10, 12 against FP64 p = 15 (-1: not measured); p_chosen the order it chose (0: none); the graph replay
 * times (ms) of the batch on test charges with the sweep off and on (-1: not timed); sweep_on whether the
 * sweep is in use. */
fmm_status fmm_batch_tune_info(fmm_batch batch, double *p_err, int *p_chosen, double *ms_sweep_off, double *ms_sweep_on,
                               int *sweep_on);

/* The deepest level of box i and the tile brick of its tensor-core M2L (0s without the tensor-core path). */
fmm_status fmm_batch_brick_info(fmm_batch batch, int i, int *level, int *bx, int *by, int *bz);

/*
 * One evaluation of every box.  pos[i] (double[N_i][3]), q[i] (double[N_i]),
 * is_solute[i] (uint8_t[N_i]): DEVICE pointers, which must stay valid and
 * unchanged in place between calls that reuse them.  lambda_c: host double[nbox]
 * (NULL: all 0).  Outputs (host double[nbox], each nullable): e_total, e_uv,
 * v_lambda = e_total - lambda_c e_uv, dv_dlambda = -e_uv (with the soft-core
 * near field on: see fmm_batch_set_softcore).  Synchronises.
 *
 * The first call runs the boxes through the streams and then records the whole
 * batch as a CUDA graph; later calls with the same pointers replay it and
 * check every box's solute count against the recorded one, falling back to
 * the stream path (and recording again) when one differs.  Returns the first
 * error among the boxes (FMM_ERR_NONFINITE, FMM_ERR_TIMEOUT, ...), after
 * filling the outputs of all boxes.
 */
fmm_status fmm_batch_lambda_energies(fmm_batch batch, const double *const *pos, const double *const *q,
                                     const uint8_t *const *is_solute, const double *lambda_c, double *e_total,
                                     double *e_uv, double *v_lambda, double *dv_dlambda);

/*
 * Soft-core near field for every box (FMM_OPT_SOFTCORE on each plan): c (0 = off), A (A), alpha.  With it
 * on, the solute-solvent near-field pairs of box i interact through (alpha lambda_i A^c + r^c)^(1/c), so
 * with E_uv^sc = E_uv - NF_uv + NF_sc(lambda_i) (Eq. Vswucheme with the softened NF pairs):
 *     v_lambda   = e_total - e_uv + (1 - lambda_i) E_uv^sc,
 *     dv_dlambda = -E_uv^sc + (1 - lambda_i) dNF_sc/dlambda.
 * Errors: FMM_ERR_INVALID_ARG for c outside 0..12 or, with c > 0, A or alpha not finite and positive.
 */
fmm_status fmm_batch_set_softcore(fmm_batch batch, int c, double A, double alpha);

/* Depth and order of box i, and how many calls replayed the graph or ran the
 * stream path (each nullable). */
fmm_status fmm_batch_info(fmm_batch batch, int i, int *depth, int *p, int64_t *replays, int64_t *enqueued);

/* enable = 0 drops the recorded graph and keeps to the stream path; 1 (the
 * default) allows recording. */
fmm_status fmm_batch_set_graph(fmm_batch batch, int enable);

/*
 * Persistent sweep (mixed precision).  The M2L of Eq. Lcoeffdef with the fused
 * L2L, on every level that runs on CTA pairs (full 128-target tiles, an even
 * number per parity class: level 4 and deeper), is done for all boxes of the
 * batch in ONE launch of persistent CTA pairs that pull work items from a
 * device queue: per (box, level) the split of the parent level's local
 * expansion, the tile pairs of the M2L, and the sum of the offset groups.  The
 * items are queued level by level, so each depends only on earlier ones; a pair
 * waits (bounded by FMM_BATCH_OPT_WAIT_BUDGET_NS, globaltimer) until the stage
 * it depends on has counted all its items done.  The launch is part of the
 * recorded graph.  Boxes whose order differs from the first box taking part,
 * or whose tree has no such level, keep their per-level launches.  Results are
 * bitwise those of the per-level launches (the same tile arithmetic, offset
 * groups and summation order).  A dependency wait that runs out stops the
 * launch: every box of the sweep then reports FMM_ERR_TIMEOUT, and the next
 * call starts afresh.
 */
enum {
    FMM_BATCH_OPT_SWEEP = 1,           /* ival 1 (default) / 0: the persistent sweep on / per-level launches */
    FMM_BATCH_OPT_WAIT_BUDGET_NS = 2,  /* ival 1000 .. 1e10: budget of each dependency wait (default 2e9) */
    FMM_BATCH_OPT_INJECT_STALL = 3,    /* ival 0 / 1, a test hook for the timeout path: with 1 the first
                                          tile pair's dependency asks for one item more than its stage has,
                                          so its wait runs out */
    FMM_BATCH_OPT_SWEEP_PAIRS = 4      /* ival 0 .. 4096: CTA pairs of the sweep launch (0, the default: as
                                          many as can be resident); fewer leave SMs to the boxes' near-field
                                          and solute-pass work, which does not depend on the sweep */
};

/* Set a batch option (the keys above; dval unused).  Drops the recorded graph.
 * Errors: FMM_ERR_INVALID_ARG for an unknown key or a value out of range. */
fmm_status fmm_batch_set_option(fmm_batch batch, int key, int64_t ival, double dval);

/* Boxes the sweep covers (0 with the sweep off or when no box takes part) and,
 * when first_level is not NULL (int[nbox]), each box's first sweep level (0:
 * not in the sweep). */
fmm_status fmm_batch_sweep_info(fmm_batch batch, int *boxes, int *first_level);

/* Release the batch, its plans and streams.  Accepts NULL. */
void fmm_batch_destroy(fmm_batch batch);

/*
 * Background-charge terms without a plan and without allocating anything.
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: a host application or plug-in whose device
 * memory all belongs to another allocator or a fixed budget, and loops that
 * cannot pay for the synchronisation an allocation may cause.
 *
 * pos: device double[N][3]; q: device double[N]; box: cell side (A);
 * kappa: the splitting parameter in 1/A that the plan would use (<= 0 selects
 * 2 / box, the plan default).  out: device double[8], written with
 *   {Q, mu_x, mu_y, mu_z, S2 = sum q r^2, charged, quad_surface, dipole_surface}
 * where the last three equal the fmm_energy_terms fields of the same names for
 * a plan with the conducting boundary (FMM_BOUNDARY_CONDUCTING, the default);
 * a caller using the vacuum boundary drops out[7].  Coordinates are wrapped
 * into [0, box) as the plans do.  Work is enqueued on `stream` (a
 * cudaStream_t; NULL = legacy default stream); nothing is synchronised, so no
 * device-side status comes back: a NaN or Inf charge or coordinate makes the
 * affected outputs non-finite instead of returning FMM_ERR_NONFINITE.
 *
 * The only scratch is a file-scope device array of 80 KiB that every GPU
 * loading the library keeps until the process exits; it bounds N to
 * 4,194,304 charges (larger N: FMM_ERR_INVALID_ARG, nothing launched).  The
 * first call on each device looks up that array's device address (a
 * runtime query); later calls reuse it.  All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads)
 * race, so serialise them.  Other errors: FMM_ERR_INVALID_ARG for null
 * pointers, N < 1 or a non-finite or non-positive box; FMM_ERR_CUDA if the
 * lookup or a launch fails.
 */
fmm_status fmm_background_terms_noalloc(const double *pos, const double *q, int64_t N, double box, double kappa,
                                        double *out, void *stream);

/* Static string for a status code. */
const char *fmm_status_string(fmm_status status);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
