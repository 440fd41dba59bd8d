/*
 * pkifmm — periodic kernel-independent FMM on one GB300 (sm_103a).
 *
 * C ABI of the evaluation path of "Flexibly imposing periodicity in kernel
 * independent FMM: a Multipole-To-Local operator approach" (Yan & Shelley).
 *
 * The problem (Sec. 2.2, Eq. (pfmmDef)): given S sources y_s with densities
 * phi_s and T targets x_t in the cubic box B0 = [lo, lo+L)^3, evaluate
 *     q_t = sum_s sum_{p in P} K(x_t, y_s + p) phi_s
 * where P is the lattice of periodic vectors along the periodic axes and K is
 * the Laplace kernel 1/r (k = 1) or the Stokes velocity kernel
 * (1/8pi)(I/r + r r^T/r^3) (k = 3, viscosity 1) of Eq. (kexamples).  The
 * source image that coincides with a target (the p = 0, s = t term) is
 * excluded.  The sum is split (Eq. (pfmmSplit)) into a near field over B0 and
 * its adjacent images, evaluated by KIFMM on one octree of B0, and a far
 * field carried by one precomputed operator applied to the root's upward
 * equivalent density (Algorithm 2, Stage 2 c), folded into the downward pass
 * (the L2L option of Sec. 4).
 *
 * Conventions that make the periodic sum unique (Sec. 2.2 Eq.
 * (compatcondition), Sec. 3.3, Sec. 3.4):
 *   Laplace, any periodicity: charges must be neutral;
 *   Stokes SP/DP: net force must be zero;
 *   DP (x, y periodic, z free; Sec. 3.3): the k_par = 0 (sheet) part of K^P
 *     is fixed up to a z-independent constant, which cancels by the above;
 *   Stokes TP: a net force is allowed, zero mean flow (Hasimoto, k = 0 removed).
 *   Laplace TP: k = 0 removed (zero mean potential).
 *
 * Memory: every array argument of pkifmm_evaluate is a DEVICE pointer owned
 * by the caller, contiguous, binary64.  pkifmm_evaluate_host takes HOST
 * pointers instead and copies inside the call.  The library owns its
 * operators (allocated by pkifmm_plan_create) and its workspace (grown on
 * demand by evaluate, freed by pkifmm_plan_destroy).
 *
 * Threading: a plan may be used by one host thread at a time.
 * Errors: every int-returning call returns PKIFMM_OK (0) or a negative code;
 * pkifmm_strerror gives a message.  A failed evaluate leaves pot undefined
 * and the plan usable.
 */
#ifndef PKIFMM_H
#define PKIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pkifmm_plan_s *pkifmm_plan;

/* Kernels, Eq. (kexamples): source/target dimension k = 1 and 3 (Sec. 2.3).
 * Two more target quantities (Sec. 2.3 names kernels whose source and target
 * dimensions differ, e.g. the Stokes pressure kernel R^3 -> R):
 *   PKIFMM_LAPLACE_FIELD   Laplace charges (k_s = 1); each target receives
 *                          k_t = 4 values: the potential and its gradient
 *                          (d/dx, d/dy, d/dz) with respect to the target.  The
 *                          translations are those of the Laplace kernel; only
 *                          the target evaluations differ.
 *   PKIFMM_STOKES_PRESSURE Stokes forces (k_s = 3); each target receives
 *                          k_t = 4 values: the velocity and the pressure
 *                          p = sum f.r/(4 pi r^3) (viscosity 1).  The pressure
 *                          is the Laplace potential of dipoles f at the
 *                          sources, summed in the same call by a second KIFMM
 *                          with Laplace translations (dipole kernel at the
 *                          sources, monopole equivalent densities).  Needs zero
 *                          net force for every periodicity (each force
 *                          component neutral); TP pressure has zero mean.
 * Densities are [nrhs][S][k_s], potentials [nrhs][T][k_t]; k_s = k_t = k for
 * PKIFMM_LAPLACE and PKIFMM_STOKES. */
enum { PKIFMM_LAPLACE = 0, PKIFMM_STOKES = 1, PKIFMM_LAPLACE_FIELD = 2, PKIFMM_STOKES_PRESSURE = 3 };

/* Arithmetic of the evaluation:
 * FP64  — every stage in binary64 (accuracy reference path);
 * MIXED — kernel sums (P2P, S2M, L2T, W, X) in binary32 on leaf-local
 *         coordinates with compensated accumulation; M2L on the tensor cores
 *         (tcgen05) as scaled split-fp16 pairs (three products) accumulated
 *         in binary32; the other translations in binary32; the root periodic
 *         operator and its check-to-equivalent solve in binary64.  Needs an
 *         sm_103 GPU. */
enum { PKIFMM_FP64 = 0, PKIFMM_MIXED = 1 };

/* OR-ed into `precision` of pkifmm_plan_create: build Stage 1 on the host
 * (OpenMP) instead of the device. */
enum { PKIFMM_PRECOMPUTE_HOST = 0x100 };

enum {
    PKIFMM_OK = 0,
    PKIFMM_ERR_INVALID_ARG = -1,  /* bad argument (sizes, NULL, NaN coordinate) */
    PKIFMM_ERR_OUT_OF_BOX = -2,   /* a point outside [lo, lo+L) along a free axis */
    PKIFMM_ERR_NOT_NEUTRAL = -3,  /* compatibility condition violated */
    PKIFMM_ERR_CUDA = -4,         /* a CUDA runtime call failed */
    PKIFMM_ERR_OOM = -5,          /* device or host allocation failed */
    PKIFMM_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    PKIFMM_ERR_CACHE = -7,        /* operator cache unreadable / unwritable */
    PKIFMM_ERR_UNSUPPORTED = -8   /* combination not built (MIXED without tcgen05) */
};

/* Build a plan: Algorithm 2, Stage 1 (precompute), Sec. 2.2-2.3.
 *   kernel         PKIFMM_LAPLACE or PKIFMM_STOKES
 *   periodic_axes  bit 0 = x, bit 1 = y, bit 2 = z; 0 = free space.
 *                  Every mask is built: 0 (free space), one axis (SP: 1,
 *                  2 or 4), two axes (DP: 3, 5, 6), 7 (TP).  DP in (x, z)
 *                  or (y, z) runs the (x, y) operators in a frame whose
 *                  axes are permuted so the free axis is last (points,
 *                  vector densities and vector results are carried into
 *                  it and back; the tree and list exports are in that
 *                  frame).
 *   box_lo, box_len  B0 = [box_lo, box_lo + box_len)^3 (host pointer, 3 doubles)
 *   p              points per edge of the equivalent/check surfaces (Sec. 2.2,
 *                  n = 6(p-1)^2 + 2), 4 <= p <= 16
 *   ell            near-field layers of images (Eq. (pfmmSplit)), >= 1
 *   leaf_max       s: a box splits while it holds more than s sources or
 *                  more than s targets (Sec. 2.2 notation)
 *   depth_max      deepest octree level, 1..15
 *   precision      PKIFMM_FP64 or PKIFMM_MIXED, optionally | PKIFMM_PRECOMPUTE_HOST
 *   nrhs           density vectors evaluated together on one geometry (>= 1)
 *   cache_dir      directory for the operator cache (NULL: no cache)
 * Stage 1 runs on the current CUDA device by default (binary64 kernels: the
 * surface matrices, the one-sided Jacobi SVD, the M2M / L2L products, the
 * K^{P,F} table of the root operator), or on the host with
 * PKIFMM_PRECOMPUTE_HOST; both give the same operators up to rounding.  The
 * operators stay on the current device.  On success *out owns them. */
int pkifmm_plan_create(pkifmm_plan *out, int kernel, unsigned periodic_axes,
                       const double box_lo[3], double box_len, int p, int ell,
                       int leaf_max, int depth_max, int precision, int nrhs,
                       const char *cache_dir);

/* A finite array of cells (Sec. 4: the far-field operator can describe other
 * geometries, e.g. a channel of finite length): B0 and its copies shifted by
 * n box_len along `axis` (0, 1, 2), |n| <= nimg (nimg >= 1), free in the other
 * directions.  The adjacent copies are the root's colleagues in the octree
 * (as for one periodic axis); the root operator is the plain free-space sum
 * over the copies 2 <= |n| <= nimg (it does not depend on ell).  Every point
 * must lie inside B0 (OUT_OF_BOX otherwise, no wrapping); no compatibility
 * condition applies.  Other arguments and errors as pkifmm_plan_create. */
int pkifmm_plan_create_finite(pkifmm_plan *out, int kernel, int axis, int nimg,
                              const double box_lo[3], double box_len, int p, int ell,
                              int leaf_max, int depth_max, int precision, int nrhs,
                              const char *cache_dir);

/* Evaluate potentials (Algorithm 2, Stage 2) on `cuda_stream` (a
 * cudaStream_t, NULL = legacy default stream).  Device pointers:
 *   src_xyz [S][3]            source positions
 *   dens    [nrhs][S][k_s]    source densities phi
 *   trg_xyz [T][3]            target positions (may equal src_xyz)
 *   pot     [nrhs][T][k_t]    output potentials q, overwritten
 * Positions along periodic axes may lie anywhere (they are wrapped); along
 * free axes they must lie in [lo, lo+L).  S, T >= 0 (S = 0 or T = 0 gives
 * zeros).  The call synchronises with the stream a few times while it sizes
 * the octree; it returns after enqueuing the last kernel. */
int pkifmm_evaluate(pkifmm_plan plan, int64_t S, const double *src_xyz,
                    const double *dens, int64_t T, const double *trg_xyz,
                    double *pot, void *cuda_stream);

/* Same as pkifmm_evaluate with HOST arrays: copies inputs to the device,
 * evaluates, copies pot back and synchronises the stream before returning. */
int pkifmm_evaluate_host(pkifmm_plan plan, int64_t S, const double *src_xyz,
                         const double *dens, int64_t T, const double *trg_xyz,
                         double *pot, void *cuda_stream);

/* Many independent problems in one evaluation (a batch), e.g. a set of
 * unit cells of different sizes sharing kernel, periodicity, box and p
 * (each problem is the problem of Sec. 2.2 on its own).  Problem j owns
 * sources src_off[j] .. src_off[j+1]-1 and targets trg_off[j] ..
 * trg_off[j+1]-1 of the concatenated arrays:
 *   src_off, trg_off  HOST arrays of nprob + 1 non-decreasing int64,
 *                     src_off[0] = trg_off[0] = 0; S = src_off[nprob],
 *                     T = trg_off[nprob]
 *   src_xyz, dens, trg_xyz, pot  DEVICE arrays laid out as in
 *                     pkifmm_evaluate for S sources and T targets
 *                     (dens [nrhs][S][k_s], pot [nrhs][T][k_t]).
 * All problems are evaluated together: one forest with one root per
 * problem (problem index above the Morton key), every stage one pass over
 * all problems' boxes; no interaction crosses problems.  The compatibility
 * condition is checked per problem (NOT_NEUTRAL if any problem violates
 * it).  nprob >= 1 with nprob <= 2^(63 - 3 depth_max); otherwise
 * INVALID_ARG.  Results equal nprob separate pkifmm_evaluate calls up to
 * rounding. */
int pkifmm_evaluate_batched(pkifmm_plan plan, int nprob, const int64_t *src_off,
                            const int64_t *trg_off, const double *src_xyz,
                            const double *dens, const double *trg_xyz, double *pot,
                            void *cuda_stream);

/* How the far field of the images beyond the near layers reaches the targets
 * (Algorithm 2, Stage 2):
 *   PKIFMM_FAR_L2L     (default) the root's downward equivalent density is
 *                      passed down the tree by L2L with the rest (the L2L
 *                      option of Sec. 4);
 *   PKIFMM_FAR_DIRECT  step d: it is evaluated directly at every target,
 *                      q_F = K(x_t, y^{B0,d}) phi^{B0,d}, in binary64, O(T p^2).
 * Both give the same potentials up to the method's error.  Applies to later
 * evaluations; INVALID_ARG for other modes.  No effect in free space. */
enum { PKIFMM_FAR_L2L = 0, PKIFMM_FAR_DIRECT = 1 };
int pkifmm_plan_set_far_field(pkifmm_plan plan, int mode);

/* Leaf-size autotuner (the paper fixes s by hand, Sec. 3.5; no counterpart).
 * For each candidate leaf size s (candidates[0..ncand-1], each >= 1) the
 * plan evaluates the given batch (arguments as pkifmm_evaluate_batched) once
 * to warm up and then `reps` times, timing each call on the host clock
 * around the call plus a stream synchronisation; the fastest candidate
 * becomes the plan's leaf size and is written to *best_out, the per
 * candidate minimum times (ms) to ms_out[0..ncand-1] (nullable).  pot holds
 * the last evaluation's result.  Operators do not depend on s, so nothing
 * is recomputed.  On error the plan keeps its previous leaf size. */
int pkifmm_autotune_leaf(pkifmm_plan plan, int nprob, const int64_t *src_off,
                         const int64_t *trg_off, const double *src_xyz,
                         const double *dens, const double *trg_xyz, double *pot,
                         const int *candidates, int ncand, int reps, int *best_out,
                         double *ms_out, void *cuda_stream);

/* Per-stage device times (ms) of the last evaluate, in this order:
 * 0 keys+sort, 1 tree+lists, 2 upward (S2M, M2M), 3 root periodic operator,
 * 4 M2L (V list), 5 X list + downward (C2E, L2L), 6 leaves (L2T, W, P2P),
 * 7 total, 8 the tensor-core M2L kernel alone (MIXED plans; else 0).
 * Writes min(max, 9) values; returns that count (or an error).  Waits for
 * the last evaluate's work to finish. */
int pkifmm_last_stage_times(pkifmm_plan plan, double *ms, int max);

/* Counts describing the octree of the last evaluate:
 * 0 boxes, 1 leaves, 2 depth, 3 |U| entries, 4 |V| entries, 5 |W|, 6 |X|,
 * 7 source-target pairs of the U list.  Writes min(max, 8) values. */
int pkifmm_tree_stats(pkifmm_plan plan, int64_t *out, int max);

/* Copy the octree and interaction lists of the last evaluate to host arrays
 * (for verification).  Boxes are numbered level by level, Morton order within
 * a level (octant bits x = 1, y = 2, z = 4).  Any pointer may be NULL.
 *   level[nbox], pos[nbox][3] (integer position at its level), parent[nbox]
 *   (-1 for the root), src_range[nbox][2], trg_range[nbox][2] (into the
 *   sorted order), src_perm[S] / trg_perm[T] (sorted -> input index).
 * Lists (name 'U','V','W','X'): list_ptr[nbox+1] CSR offsets, list_box[n]
 * source box, list_shift[n][3] periodic image in {-1,0,1}.  pkifmm_list_export
 * returns n (>= 0, the entry count; call with NULL arrays to size them) or a
 * negative error. */
int pkifmm_tree_export(pkifmm_plan plan, int32_t *level, int32_t *pos, int32_t *parent,
                       int64_t *src_range, int64_t *trg_range, int64_t *src_perm,
                       int64_t *trg_perm);
int pkifmm_list_export(pkifmm_plan plan, char name, int64_t *list_ptr, int32_t *list_box,
                       int8_t *list_shift);

/* Singular values (descending) of the check-to-equivalent matrix
 * A_ij = K(x_i^{B0,d}, y_j^{B0,d}) of Sec. 2.3 / Table 1: check points on a
 * cube of edge 1.05, equivalent points on a cube of edge 2.95, p points per
 * edge.  Host-only (no GPU); s_out has k*(6(p-1)^2+2) entries. */
int pkifmm_surface_singular_values(int kernel, int p, double *s_out);

/* Max |A x - b| of the backward-stable solve x = V (S^+ (U^T b)) of Sec. 3.1
 * and Appendix B for b = 1 (all ones), A as above.  Host-only. */
int pkifmm_backward_error(int kernel, int p, double *err_out);

/* Root far-field operator (host-only, row-major [kn][kn], unit box):
 * M = K^{P,F}_ell(x^{B0,d}, y^{B0,u}) + sum_{1 < |p|_inf <= ell} K(x^{B0,d}, y^{B0,u} + p)
 * i.e. the right-hand side of Eq. (M2Lsolve) with the images of layers
 * 2..ell folded in, so it maps the root's upward equivalent density to the
 * far-field check potential on the root's downward check surface (edge
 * 1.05).  K^{P,F} = K^P - sum_{|p|<=ell} K(., . + p) (Sec. 2.2).  Same
 * periodicities as pkifmm_plan_create (non-zero). */
int pkifmm_root_operator(int kernel, unsigned periodic_axes, int p, int ell, double *m_out);

/* Stable Morton ordering of points without allocating any device memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc -- a process whose device memory is entirely owned by another
 * framework's memory pool, a real-time loop that forbids allocation after
 * start-up, or host code running where CUDA allocation calls are not
 * permitted.  It computes what pkifmm_evaluate's first step computes for its
 * sources: points normalised to [box_lo, box_lo + box_len)^3, wrapped along
 * periodic axes, keyed by their cell at `depth` (Morton order, octant bits
 * x = 1, y = 2, z = 4) and sorted stably, ties in input order.
 *   xyz   DEVICE [n][3] binary64 positions (caller-owned)
 *   perm  DEVICE [n] int32 output: perm[i] = input index of the i-th point
 *   n     0 <= n <= 131072; larger n returns PKIFMM_ERR_INVALID_ARG before
 *         any GPU work (the scratch is fixed)
 *   depth 1..15; box_lo is a host pointer; cuda_stream as in pkifmm_evaluate
 * Scratch: one fixed array of about 6 MB in device memory, defined with the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on a device (and the first after a device reset)
 * looks up its address on that device (cudaGetSymbolAddress); make that first
 * call before any stream capture.  Every call shares the array and leaves its
 * contents behind, so calls whose GPU work overlaps (different streams or
 * threads at once) race and give wrong results.  Each call copies its error
 * flags back to the host and synchronises `cuda_stream` before it returns.
 * Errors as pkifmm_evaluate (OUT_OF_BOX for a point outside a free axis,
 * INVALID_ARG for a non-finite coordinate, CUDA with the failing step in
 * pkifmm_last_error_message). */
int pkifmm_morton_order_noalloc(int64_t n, const double *xyz, const double box_lo[3], double box_len,
                                unsigned periodic_axes, int depth, int32_t *perm, void *cuda_stream);

/* Host-only view of the root operator of a finite array of cells (see
 * pkifmm_plan_create_finite): m_out [kn][kn], the free-space kernel from the
 * upward equivalent surface of B0 to its downward check surface summed over
 * the copies 2 <= |n| <= nimg along `axis`. */
int pkifmm_root_operator_finite(int kernel, int axis, int nimg, int p, double *m_out);

/* Stage 1 alone (Algorithm 2; Sec. 2.2-2.3, 3.1), without a plan, for
 * comparing and timing the host (where = 0) and device (where = 1) builds.
 * kernel, periodic_axes, p, ell, precision as for pkifmm_plan_create (the
 * precision selects the SVD cut-off, as for a plan).  Host output
 * buffers, each may be NULL:
 *   s_out      [kn]          singular values of the upward check-to-equivalent
 *                            matrix K(1.475 g, 0.525 g), descending
 *   m2m_out    [8][kn][kn]   child-octant -> parent upward densities
 *   l2l_out    [8][kn][kn]   parent -> child-octant downward densities
 *   root_out   [kn][kn]      root far-field operator (periodic masks only)
 *   seconds_out              wall time of the build (the device build counts
 *                            its transfers, not CUDA context creation)
 *   phases_out [4]           device build only: seconds of the SVD, of the
 *                            M2M / L2L products, of the root table, then the
 *                            number of Jacobi sweeps
 * kn = 6(p-1)^2 + 2 for Laplace, 3 times that for Stokes.  Nothing is cached. */
int pkifmm_precompute_operators(int kernel, unsigned periodic_axes, int p, int ell,
                                int precision, int where, double *s_out, double *m2m_out,
                                double *l2l_out, double *root_out, double *seconds_out,
                                double *phases_out);

void pkifmm_plan_destroy(pkifmm_plan plan);
const char *pkifmm_strerror(int code);

/* Detail message of the last failed call on this host thread (library-owned
 * string, valid until the next failing call on the thread). */
const char *pkifmm_last_error_message(void);

/* Total number of CUDA kernels this library has launched in this process
 * (all plans and threads).  The difference across a region counts the
 * launches inside it. */
int64_t pkifmm_launch_count(void);

/* Dimension the plan's V-list M2L works in (Sec. 2.2, the M2L translation):
 * kn = k (6(p-1)^2 + 2) when it applies the 316 dense check-form operators
 * K_o (FP64 plans, and MIXED plans where a shared basis would not cut the
 * tensor-core work by 30%), or r < kn when the MIXED path applies
 * C_o = Ub^T K_o Ub in the shared basis Ub of the stacked operators (r columns;
 * see include notes of pkifmm_plan_create).  Negative on a NULL plan. */
int pkifmm_m2l_rank(pkifmm_plan plan);

/* 1 if MIXED plans run their M2L on the tensor cores of the current device
 * (tcgen05, sm_103), else 0 (MIXED plans then fail with UNSUPPORTED). */
int pkifmm_m2l_tensor_core_enabled(void);

#ifdef __cplusplus
}
#endif
#endif /* PKIFMM_H */
