/*
 * nbody.h -- C ABI of the GB300 periodic treecode force path.
 *
 * The operations follow the N-body method of Sec. 2.1 of the paper ("2HOT"):
 * particles get Morton keys and are sorted by them (the key order maps 3-D
 * space to a line and the sort doubles as the domain decomposition), the
 * keys imply an oct-tree whose cells are found through a hash of their keys,
 * cells carry truncated multipole expansions, a multipole acceptance test
 * decides between using a cell's expansion and opening it, sinks are
 * bundled into groups that share one interaction list, and near-leaf
 * interactions are direct particle-particle sums; boundaries are periodic.
 * Sec. 2.1 also names a symplectic integrator; the kick-drift-kick step in
 * comoving coordinates is provided here, with its adjoint.
 *
 * Conventions for every entry point:
 *   - Units: each box is the unit periodic cube; positions are FP64 in [0,1)
 *     (finite values outside are wrapped; NaN or Inf is NBODY_EINVAL), G = 1, accelerations are in units of
 *     G * (unit mass) / (box length)^2.  With masses summing to 1 per box the
 *     mean density is 1.
 *   - Layout: arrays are structure-of-arrays in the caller's particle order:
 *     pos = [x_0..x_{n-1}, y_0..y_{n-1}, z_0..z_{n-1}], likewise for momenta
 *     and accelerations.  Pointers marked _dev are device pointers on the
 *     current CUDA device.
 *   - Ownership: the caller owns every array it passes and must keep the
 *     position, momentum and mass arrays it hands to a tree alive while the
 *     tree is used.  The library owns the tree handle and its scratch memory
 *     (freed by nbody_tree_free) and a per-device table of the periodic image
 *     field (freed at process exit).
 *   - Streams: work is enqueued on the given stream.  By default each call
 *     ends with a blocking read of a 4-byte device status word so that
 *     device-side errors (overflow, bounded waits that ran out) come back as
 *     return codes; NBODY_FLAG_ASYNC in params.flags skips that read and the
 *     status can be fetched later with nbody_check.
 *   - Errors: 0 on success, a negative NBODY_E* code otherwise; no entry
 *     point throws or exits.  nbody_strerror gives a message.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nbody_stream_t; /* a cudaStream_t; NULL = default stream */

enum {
  NBODY_OK = 0,
  NBODY_EINVAL = -1,    /* bad argument (null pointer, n <= 0, eps <= 0, ...) */
  NBODY_ENOMEM = -2,    /* device allocation failed */
  NBODY_ECUDA = -3,     /* a CUDA runtime call failed */
  NBODY_EOVERFLOW = -4, /* a fixed-capacity device buffer would overflow */
  NBODY_ETIMEOUT = -5,  /* a bounded device-side wait ran out */
  NBODY_ENOTSUP = -6,   /* parameter combination not supported */
  NBODY_ERANGE = -7     /* size beyond the fixed maximum of an allocation-free entry point */
};

enum { NBODY_MIXED = 0, NBODY_FP64 = 1 };
enum {
  NBODY_FLAG_ASYNC = 1,
  /* opening test with d measured from the cell's faces to the group box
   * (box-to-box distance) instead of from the cell centre: a stricter test
   * at the same theta (see nbody_params.theta) */
  NBODY_FLAG_MAC_EDGE = 2,
  /* uniform-background terms (Sec. 2.1's background subtraction for
   * near-uniform states): every cell used through its expansion also adds
   * the next even order of the field of a cube of the box's mean density
   * filling it (order 4 after expansions of order 0 and 2, order 6 after
   * order 4; Newtonian kernel), i.e. the truncation error of the cell's
   * uniform share, which dominates the expansion error when the density is
   * nearly uniform.  Orders 1 and 3 reject the flag (NBODY_EINVAL). */
  NBODY_FLAG_BACKGROUND = 4,
  /* softening by Dehnen's compensating K1 kernel (the kernel Sec. 2.1 names)
   * instead of Plummer's: a direct pair at r = |d| gets a = m d f(r) with
   * f = 1/r^3 from r >= eps on (exactly Newtonian) and, for x = r/eps < 1,
   * f = (175/16 - (147/8) x^2 + (135/16) x^4)/eps^3, the enclosed mass over
   * r^3 of the density 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2) (the kernel
   * 1 - x^2 with the factor that makes its second moment vanish).  Cell
   * expansions then use the Newtonian kernel 1/|R|.  The reverse mode
   * (nbody_forces_vjp, nbody_kdk_adjoint) returns NBODY_ENOTSUP with it. */
  NBODY_FLAG_K1 = 8,
  /* dual (cell-group) interactions, the source-sink form of the traversal in
   * Sec. 2.1: an accepted cell C of side s_C whose centre lies farther than
   * (s_C + s_G)/theta from the centre z of the group's bounding box (s_G its
   * largest side; integer units of 2^-23, the threshold floor(S^2/theta^2)
   * in IEEE double) is not expanded at every sink: one local expansion per
   * (cell, group), L_k = sum_n ((-1)^|n|/n!) M_n d^(n+k) g(z - c*) with
   * 1 <= |k| and |n| + |k| <= order + 1 (the derivative orders of the
   * expansion at a sink), is accumulated per group and evaluated once per
   * sink, a_k = sum_{|m| <= order} (x - z)^m / m! L_(m + e_k).  Orders 1..4,
   * NBODY_MIXED, not with NBODY_FLAG_BACKGROUND (else NBODY_ENOTSUP); the
   * reverse mode returns NBODY_ENOTSUP with it. */
  NBODY_FLAG_DUAL = 16,
  /* periodic images by near replicas and a far-lattice expansion (Sec.
   * 2.1's periodic boundary conditions: a multipole local expansion of order
   * p = 8).  The walk visits every cell at each of the 125 images n,
   * |n|_inf <= 2, of the box (the acceptance test per image; cells of any
   * level may be accepted), and the images beyond act through one local
   * expansion about the box centre c0 of order 8: L_k = sum_n ((-1)^|n|/n!)
   * M_n T_(k+n), |k| + |n| <= 8, with the box's moments M about c0 and T the
   * derivatives at 0 of the periodic potential of a unit mass with the
   * uniform background less its near images' -1/|r - n|; every sink adds
   * a = -sum_{|u| <= 7} d^u/u! L_(u + e_k), d = x - c0.  Against the exact
   * Ewald sum the far lattice errs by about 3e-7 (median, forces).  Needs
   * ewald_order = 0 (else NBODY_EINVAL); ewald_grid - 1 is then the level
   * of the cells no group straddles.  Fewer than 2^25 cells; the reverse
   * mode returns NBODY_ENOTSUP with it. */
  NBODY_FLAG_REPLICAS = 32
};
/* flags bits 8..11: walk launch variant + 1 to use instead of the autotuned
 * one (0 = autotune).  Mixed precision has variants 0..3 (one M2P per
 * instruction stream with 8 warps x 2 or 4 x 4 blocks per SM; two M2P at
 * once in packed FP32 pairs, 8 x 2 or 4 x 4; with NBODY_FLAG_DUAL the second
 * is packed with 4 x 3); FP64 has only variant 0.  Every variant computes
 * the same interactions; results differ by the summation order only. */
#define NBODY_FLAG_WALK_VARIANT(v) (((v) + 1) << 8)

typedef struct {
  double eps;       /* Plummer softening length, box units (> 0); per-box
                       values may be given to nbody_build_tree_batched */
  double theta;     /* opening angle of the multipole acceptance test: a cell
                       of side s is expanded for a group when s / d < theta,
                       d the distance from the cell centre (or, with
                       NBODY_FLAG_MAC_EDGE, from the cell's faces) to the
                       group's bounding box, in integer units of 2^-23 */
  int order;        /* multipole order p of the cell expansions, 0..4 */
  int n_leaf;       /* cells with more particles are split (1..64) */
  int n_group;      /* sinks per group, 1..32 */
  int n_direct;     /* accepted cells with <= n_direct particles are summed
                       directly (0..n_leaf) */
  int lmax;         /* deepest tree level, 2..21 */
  int ewald_order;  /* order of the image-field local expansion, 0..5
                       (0 = no periodic images) */
  int ewald_level;  /* level of the fixed source cells of the image field */
  int ewald_grid;   /* image-field expansion points lie on the lattice
                       2^-ewald_grid; groups never straddle a cell of level
                       ewald_grid - 1 */
  int precision;    /* NBODY_MIXED (FP32 interactions, FP64 positions and
                       moments) or NBODY_FP64 (FP64 throughout) */
  int flags;        /* NBODY_FLAG_* */
  double box_len;   /* side L of the periodic box (0 or 1: the unit box).
                       Positions are then in [0, L), eps is in the same
                       length unit, and accelerations (force VJPs) come back
                       as G m / L^2 (G m / L^3) for the caller's masses, G = 1:
                       the tree works on x / L.  The comoving integrator and
                       its adjoint work in box units and return NBODY_ENOTSUP
                       for a tree with L != 1 (nbody_kdk_step,
                       nbody_kdk_multistep, nbody_assign_rungs,
                       nbody_forces_active, nbody_kdk_adjoint(_acc)). */
} nbody_params;

/* Fills the defaults: eps = 1/(30*128), theta = 0.6, order = 4, n_leaf = 16,
 * n_group = 32, n_direct = 4, lmax = 21, ewald_order = 4, ewald_level = 3,
 * ewald_grid = 6, precision = NBODY_MIXED, flags = 0, box_len = 1. */
void nbody_default_params(nbody_params *p);

typedef struct {
  double p2p;          /* particle-particle interactions in the last evaluation */
  double m2p;          /* cell-particle (multipole) interactions */
  double m2l;          /* image-field cell-to-group translations */
  int64_t ncells;      /* tree cells (all boxes) */
  int64_t ngroups;     /* sink groups */
  int32_t max_level;   /* deepest level present */
  int32_t nbox;
  float ms_sort;       /* device time of keys + sort + gather */
  float ms_build;      /* tree topology, hash, groups, leaf offsets */
  float ms_upward;     /* moments */
  float ms_walk;       /* group walk with P2P and M2P */
  float ms_periodic;   /* image-field expansion and scatter to caller order */
  uint64_t decision_hash; /* order-independent checksum of every (group, cell,
                             decision) of the walk: equal trees and decisions
                             give equal sums (finite-difference checks use it) */
} nbody_stats;

typedef struct nbody_tree nbody_tree;

/*
 * Build (or rebuild) the tree of one periodic box: Morton keys, radix sort,
 * gather into key order, oct-tree topology and key hash, sink groups, leaf
 * offsets and the cell moments (Sec. 2.1: keys imply the tree; cells carry
 * truncated multipole expansions).
 *   n        number of particles (>= 1, < 2^30)
 *   pos_dev  3*n FP64 positions (SoA)
 *   mass_dev n FP32 masses, or NULL for equal masses 1/n
 *   tree     in: NULL or an existing handle to reuse (its buffers are kept
 *            when large enough); out: the handle
 * The tree keeps pointers to pos_dev and mass_dev.  A position or mass that
 * is not finite (NaN, +-Inf) makes the build return NBODY_EINVAL (with
 * NBODY_FLAG_ASYNC: the next nbody_check); a fresh handle is then not
 * returned, a reused one holds a meaningless tree until the next build from
 * finite positions.  Finite positions outside [0,1) are wrapped.
 */
int nbody_build_tree(const nbody_params *params, int64_t n, const double *pos_dev,
                     const float *mass_dev, nbody_tree **tree, nbody_stream_t stream);

/*
 * Same for nbox independent periodic boxes stored back to back: box b holds
 * particles [offsets[b], offsets[b+1]) (offsets_host: nbox+1 host int64,
 * offsets[0] = 0, non-decreasing with no empty box).  eps_host: nbox host
 * doubles (NULL = params->eps for all).  Masses NULL = 1/n_b in box b.
 */
int nbody_build_tree_batched(const nbody_params *params, int nbox, const int64_t *offsets_host,
                             const double *eps_host, const double *pos_dev,
                             const float *mass_dev, nbody_tree **tree, nbody_stream_t stream);

/*
 * Build and evaluate in one call: nbox independent periodic boxes of
 * possibly different sizes, as nbody_build_tree_batched followed by
 * nbody_forces (the batched realisations of Sec. 1's "multiple
 * realisations", each a periodic box of Sec. 2.1).
 *   box_len_host  nbox host doubles, the side L_b of box b (NULL: params->box_len
 *                 for every box); box b's positions are in [0, L_b) and
 *                 eps_host[b] (NULL: params->eps) is in the same unit
 *   acc_dev       3*n FP32 accelerations (caller order), G m / L_b^2 for the
 *                 caller's masses (NULL masses: 1/n_b per box)
 *   tree          as nbody_build_tree (NULL or a handle to reuse)
 * Errors as nbody_build_tree_batched and nbody_forces.
 */
int nbody_forces_batched(const nbody_params *params, int nbox, const int64_t *offsets_host,
                         const double *box_len_host, const double *eps_host, const double *pos_dev,
                         const float *mass_dev, float *acc_dev, nbody_tree **tree, nbody_stream_t stream);

/*
 * Accelerations of all particles of the tree (Sec. 2.1: grouped tree walk with
 * the acceptance test, multipole and direct interactions, periodic images).
 *   acc_dev  3*n FP32 (SoA, caller order), overwritten
 *   pot_dev  NULL, or n FP32 (caller order), overwritten with the potential
 *            of the same evaluation: the periodic potential in the zero-mean
 *            convention (the uniform neutralising background included),
 *            G = 1, in the caller's units (mass / length); each particle's
 *            own images and background count, its softened self pair does
 *            not.  Every interaction contributes its potential form: a
 *            direct pair -m (r^2 + eps^2)^-1/2 (Plummer) or the K1 kernel's
 *            -m (105/32 - 175/32 x^2 + 147/32 x^4 - 45/32 x^6)/eps inside
 *            eps; an accepted cell -sum_n ((-1)^|n|/n!) M_n d^n g, also
 *            under NBODY_FLAG_DUAL (the potential is the expansion form's;
 *            the accelerations stay the dual form's); the image field its
 *            local expansion's series; the background -(2 pi/3) sum m |x -
 *            x*|^2.  The potential comes from a second, scalar variant of the
 *            walk, so asking for it costs one walk or more.
 *            NBODY_ENOTSUP with ewald_order 1 (the background's potential
 *            needs the image cells' second moments).
 *   stats    NULL or filled with counts and phase times (phase times are
 *            only filled when the call synchronises)
 */
int nbody_forces(nbody_tree *tree, float *acc_dev, float *pot_dev, nbody_stats *stats, nbody_stream_t stream);

/*
 * nbody_forces with FP64 output: acc_dev is 3*n FP64 (caller order,
 * overwritten).  With precision NBODY_FP64 the accelerations are FP64
 * throughout (for FP64 finite-difference checks of the reverse mode); with
 * NBODY_MIXED they are the FP32 results widened.  Errors as nbody_forces.
 */
int nbody_forces64(nbody_tree *tree, double *acc_dev, nbody_stream_t stream);

/*
 * One kick-drift-kick step in comoving coordinates (Einstein-de Sitter,
 * p = a^2 dx/dt, dx/dt = p/a^2, dp/dt = g/a, H = H0 a^-3/2,
 * H0^2 = 8 pi / 3 for unit mean density), the global-step form of the
 * symplectic integrator cited in Sec. 2.1:
 *   p += K(a0, ah) g(x0);  x += D(a0, a1) p (wrapped);  rebuild + forces;
 *   p += K(ah, a1) g(x1);  ah = sqrt(a0 a1),
 *   K(a,b) = (2/H0)(sqrt b - sqrt a),  D(a,b) = (2/H0)(a^-1/2 - b^-1/2).
 *   pos_dev  3*n FP64, updated in place (must be the tree's positions)
 *   mom_dev  3*n FP32 momenta, updated in place
 *   acc_dev  3*n FP32: in g(x0), out g(x1)
 * A drifted position that is not finite (from a non-finite momentum or
 * acceleration) makes the step's rebuild, and so the step, return
 * NBODY_EINVAL.
 */
int nbody_kdk_step(nbody_tree *tree, double *pos_dev, float *mom_dev, float *acc_dev, double a0,
                   double a1, nbody_stream_t stream);

/*
 * Block steps (the hierarchical form of the symplectic integrator cited in
 * Sec. 2.1, Quinn et al. 1997).  A global step in ln a is cut into
 * T = 2^rmax ticks uniform in ln a (tick j at a_j = a0 exp(j ln(a1/a0)/T)); a
 * particle on rung r takes steps of S = 2^(rmax - r) ticks in kick-drift-kick
 * form: when its step starts it is kicked over the step's first half,
 * K(a_j, a_{j+S/2}); every tick all particles drift D(a_j, a_{j+1}) and the
 * tree is rebuilt; when its step ends its acceleration is recomputed (only
 * the groups holding such particles are walked) and it is kicked over the
 * second half.  Rungs stay fixed during the call.  With rmax = 0 this is
 * nbody_kdk_step.
 *
 * nbody_assign_rungs: rung of each particle from its acceleration, the
 * smallest r in [0, rmax] with 4^r >= |g| dlna^2 / (eta^2 H0^2 eps) (eps of
 * the particle's box, |g| from the FP32 acc in FP64): the step at which a
 * particle moves about eta^2 eps under g.
 *   acc_dev   3*n FP32 accelerations (caller order)
 *   eta > 0, dlna > 0 (the global step in ln a), rmax 0..7
 *   rung_dev  n int8 output (caller order)
 * nbody_forces_active: accelerations of the particles with rung >= rmin at
 * the last build's positions; the other entries of acc_dev are not written.
 * nbody_kdk_multistep: one global step a0 -> a1 (a1 > a0); pos_dev, mom_dev,
 * acc_dev as in nbody_kdk_step (acc_dev must hold every particle's
 * acceleration at the start, and holds each particle's last one at the end);
 * rung_dev n int8 in [0, rmax].
 */
int nbody_assign_rungs(nbody_tree *tree, const float *acc_dev, double eta, double dlna, int rmax,
                       int8_t *rung_dev, nbody_stream_t stream);
int nbody_forces_active(nbody_tree *tree, const int8_t *rung_dev, int rmin, float *acc_dev,
                        nbody_stream_t stream);
int nbody_kdk_multistep(nbody_tree *tree, double *pos_dev, float *mom_dev, float *acc_dev,
                        const int8_t *rung_dev, double a0, double a1, int rmax, nbody_stream_t stream);

/*
 * Reverse mode of one nbody_kdk_step, with g(x0) recomputed from pos0 (so the
 * step is a function (x0, p0) -> (x1, p1)).  Given the cotangents of the
 * step's outputs it returns those of its inputs:
 *   pos0_dev, mom0_dev      the state at the start of the step (not modified)
 *   lam_pos1_dev, lam_mom1_dev  3*n FP64 / FP32 cotangents of x1, p1
 *   lam_pos0_dev, lam_mom0_dev  3*n FP64 / FP32 outputs
 * The discrete decisions of the tree (topology, acceptance, groups) are held
 * fixed, so this is the exact derivative of the evaluated forces.  Uses the
 * tree's parameters; the tree is rebuilt at x0 internally (its positions are
 * then an internal copy of pos0).
 *
 * Chaining.  The step needs J(x1)^T lam_mom1 (J = d acc / d pos) and
 * J(x0)^T lam_ph; the second is kept, with x0 and lam_mom0.  When the next
 * call is the previous step of the same trajectory (its recomputed x1 equals
 * this call's x0 bit for bit and its lam_mom1 is this call's lam_mom0, which is
 * what a reverse sweep passes), the kept product is reused and that call
 * evaluates one tree instead of two.  The test is an exact comparison on the
 * device, so any other sequence of calls gives the same results, only
 * without the reuse.  The recompute uses the same FP32 kick and FP64 drift as
 * nbody_kdk_step, so a trajectory stepped by nbody_kdk_step chains.
 * Errors: EINVAL (NULL pointer, a0 or a1 <= 0), ENOTSUP (FP64 precision or
 * an image field of order > 4), plus those of nbody_build_tree.
 */
int nbody_kdk_adjoint(nbody_tree *tree, const double *pos0_dev, const float *mom0_dev, double a0,
                      double a1, const double *lam_pos1_dev, const float *lam_mom1_dev,
                      double *lam_pos0_dev, float *lam_mom0_dev, nbody_stream_t stream);

/*
 * nbody_kdk_adjoint with g(x0) supplied by the caller instead of recomputed:
 *   acc0_dev  3*n FP32, the accelerations at pos0 exactly as nbody_forces or
 *             nbody_kdk_step returned them for these positions (caller order;
 *             not modified).  The tree walk at x0 is then skipped: the call
 *             builds the tree, its moments and its image field only.
 * Results are bitwise those of nbody_kdk_adjoint when acc0 is that g(x0).
 * A checkpointed reverse sweep has g(x) of every recomputed state at hand.
 */
int nbody_kdk_adjoint_acc(nbody_tree *tree, const double *pos0_dev, const float *mom0_dev,
                          const float *acc0_dev, double a0, double a1, const double *lam_pos1_dev,
                          const float *lam_mom1_dev, double *lam_pos0_dev, float *lam_mom0_dev,
                          nbody_stream_t stream);

/*
 * Vector-Jacobian product of the force: out = (d acc / d pos)^T lam, for the
 * tree as last built (positions as given to the build).
 *   lam_dev  3*n FP32 cotangent of the accelerations (caller order)
 *   out_dev  3*n FP64, overwritten
 */
int nbody_forces_vjp(nbody_tree *tree, const float *lam_dev, double *out_dev,
                     nbody_stream_t stream);

/*
 * Device-time accounting for benchmarks.  Every build and force evaluation
 * records CUDA events on its stream into a ring (the last 64 of each are
 * kept); this call synchronises the tree's last stream, sums the phase times
 * and interaction counts since the previous reset, and optionally resets.
 */
typedef struct {
  int64_t builds;        /* tree builds timed */
  int64_t evaluations;   /* force evaluations timed */
  int64_t launches;      /* kernels launched by the library */
  double p2p, m2p, m2l;  /* interactions summed over the evaluations */
  double ms_sort, ms_build, ms_upward, ms_walk, ms_periodic; /* summed device times */
  int64_t adjoint_steps;   /* nbody_kdk_adjoint(_acc) calls */
  int64_t adjoint_reused;  /* of which reused the previous call's J(x0)^T lam_ph */
  uint64_t decision_hash;  /* sum (mod 2^64) of the evaluations' decision checksums */
  int64_t walk_variant;    /* walk launch variant the autotuner chose for this tree's
                              precision and order on this device (-1: not tuned yet) */
  double walk_tune_ms[8];  /* each variant's time in the tuning run (0: not timed) */
  double m2l_dual;         /* cell-group expansions of the dual form (NBODY_FLAG_DUAL), summed */
} nbody_timing;
int nbody_timing_read(nbody_tree *tree, nbody_timing *out, int reset);

/*
 * CIC density contrast loss of one box (the loss of the differentiable
 * trajectory; the paper has no such loss, it uses CIC grids for its power
 * spectra in Sec. 4): grid cell c of ng^3 has centre (c + 1/2)/ng,
 * delta_c = ng^3 sum_j m_j w_jc - 1, L = sum_c delta_c^2.
 *   pos_dev   3*n FP64 positions;  mass_dev  n FP32 or NULL (1/n)
 *   grid_dev  ng^3 FP64 caller workspace; holds delta on return
 *   loss_dev  one FP64 (device), the loss
 *   grad_dev  3*n FP64 dL/dpos (SoA) or NULL
 */
int nbody_cic_loss(const double *pos_dev, const float *mass_dev, int64_t n, int ng, double *grid_dev,
                   double *loss_dev, double *grad_dev, nbody_stream_t stream);

/*
 * Ends of the differentiable trajectory that are not tree work: its
 * Zel'dovich starting state and the transpose of that map (the comoving
 * growing mode of the integrator above, D = a, H0^2 = 8 pi / 3).
 * nbody_zeldovich_state: x = q + a psi wrapped into [0, 1),
 *   p = H0 a^(3/2) psi rounded to FP32.
 *   q_dev, psi_dev  3*n FP64 lattice positions and displacement field (SoA)
 *   pos_dev         3*n FP64 out;  mom_dev 3*n FP32 out
 * nbody_zeldovich_vjp: the gradient of a loss with respect to psi from the
 * cotangents of (x, p): dpsi = a lam_x + H0 a^(3/2) lam_p.
 *   lam_pos_dev 3*n FP64, lam_mom_dev 3*n FP32, dpsi_dev 3*n FP64 out
 * Both: a > 0, n >= 1, else NBODY_EINVAL; asynchronous on the stream.
 */
int nbody_zeldovich_state(int64_t n, const double *q_dev, const double *psi_dev, double a, double *pos_dev,
                          float *mom_dev, nbody_stream_t stream);
int nbody_zeldovich_vjp(int64_t n, double a, const double *lam_pos_dev, const float *lam_mom_dev,
                        double *dpsi_dev, nbody_stream_t stream);

/* Tree inspection (tests).  what: */
enum {
  NBODY_EXPORT_SORTED_KEYS = 1, /* uint64 per particle, key order */
  NBODY_EXPORT_PERM = 2,        /* uint32 per particle: original index of the i-th in key order */
  NBODY_EXPORT_CELL_KEYS = 3,   /* uint64 per cell: 1<<3l | key prefix, breadth-first order */
  NBODY_EXPORT_CELL_RANGE = 4,  /* int32 pairs (first particle, count) per cell */
  NBODY_EXPORT_CELL_LEVEL = 5,  /* int32 per cell */
  NBODY_EXPORT_MOMENTS = 6,     /* FP64 moments per cell, (order+1)(order+2)(order+3)/6 each */
  NBODY_EXPORT_GROUPS = 7,      /* int32 pairs (first particle, count) per group */
  /* FP64 derivatives d^n phi~ (|n| <= ewald_order + 1, in the moments'
   * multi-index order) of the image-field potential phi~ = phi_E + 1/|r| +
   * (2 pi/3)|r|^2 at the lattice nodes r = (i, j, k) 2^-ewald_grid,
   * 0 <= i, j, k < 2^(ewald_grid-1) + 2, node-major with k fastest: the
   * per-device table the image field reads (NBODY_EINVAL when
   * ewald_order is 0) */
  NBODY_EXPORT_IMAGE_TABLE = 8
};
/* Number of elements of an export (cells, particles, groups), or < 0. */
int64_t nbody_tree_count(const nbody_tree *tree, int what);
/* Copy an export to dst_dev (device memory sized by nbody_tree_count). */
int nbody_tree_export(const nbody_tree *tree, int what, void *dst_dev, nbody_stream_t stream);
/* Hash lookup of cell keys (1<<3l | prefix) of box 0: idx_dev[i] = cell
 * index in breadth-first order, or -1 when the key is not a cell. */
int nbody_tree_lookup(const nbody_tree *tree, const uint64_t *keys_dev, int64_t nkeys,
                      int32_t *idx_dev, nbody_stream_t stream);

/*
 * Allocation-free Morton keys + stable radix sort, for callers that cannot
 * allocate device memory at run time (another allocator owns or caps the
 * device memory, cudaMalloc's implicit synchronisation is not acceptable,
 * or the device footprint must stay fixed after set-up).  The paper has no
 * counterpart; this is the keys + sort phase of nbody_build_tree run on
 * scratch held in a file-scope device array of the library instead of
 * allocated memory.
 *   pos_dev       3*n FP64 positions (SoA), read only; finite values outside
 *                 [0,1) are wrapped, a NaN or Inf coordinate makes the call
 *                 return NBODY_EINVAL (the outputs are then meaningless)
 *   n             1 .. 2^20 particles; larger n returns NBODY_ERANGE
 *   keys_out_dev  n uint64: the Morton keys in ascending order (equal keys in
 *                 input order), caller-allocated
 *   perm_out_dev  n uint32: the input index of each sorted key, caller-allocated
 * The scratch array (about 14.7 MB) is held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up the
 * array's device address, so make it before any stream capture.  All calls
 * share the one array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  The call blocks
 * on the stream at its end to return the status of the bounded waits.
 */
int nbody_sort_keys_noalloc(const double *pos_dev, int64_t n, uint64_t *keys_out_dev,
                            uint32_t *perm_out_dev, nbody_stream_t stream);

/*
 * Fixed capacities, for steps captured in a CUDA graph (the batched
 * realisations of Sec. 2.1's "multiple realisations" run as one replayed
 * graph).  By default every build reads its cell and group counts back to the
 * host to size the cell buffers and launch grids, and stream capture cannot
 * hold that read.  After nbody_reserve the cell and group buffers are sized
 * once for max_cells and max_groups, builds keep their counts on the device
 * (the kernels read them there; grids are sized for the capacities), and a
 * build, nbody_forces and nbody_kdk_step enqueue no host synchronisation when
 * NBODY_FLAG_ASYNC is set, so they can be captured.
 *   max_cells, max_groups  capacities (both > 0); both 0 returns to counts
 *                          read back per build
 * A later build whose counts exceed a capacity writes no buffer past its end:
 * it sets the overflow status, its counts become 0 and the evaluation that
 * follows computes nothing (accelerations are left as they were); the next
 * status read (nbody_check, or any call without NBODY_FLAG_ASYNC) returns
 * NBODY_EOVERFLOW, and the caller reserves more and steps again from its own
 * saved state.  The call synchronises the stream, reallocates, rebuilds the
 * tree from the positions of its last build (which must still be valid) and
 * returns that build's status (NBODY_EOVERFLOW if it does not fit).  The
 * first nbody_forces after it (uncaptured) sizes the evaluation buffers and
 * runs the walk autotuner, so make one before capturing.  Tree statistics and
 * exports then read the counts from the device.
 */
int nbody_reserve(nbody_tree *tree, int64_t max_cells, int64_t max_groups, nbody_stream_t stream);

/*
 * Walk tile autotuner.  Times one rebuild + force evaluation of the tree's
 * current positions for every candidate pair of tile sizes -- sinks per group
 * n_group in {16, 24, 32} (the particles of a warp's shared interaction list)
 * and direct-sum threshold n_direct in {2, 4, 8, 12} (accepted cells with at
 * most that many particles are summed pairwise instead of through their
 * expansion; candidates above n_leaf are skipped) -- keeps the fastest pair
 * in the tree's parameters and rebuilds the tree with it.  Every candidate is
 * the same force definition up to which accepted cells are summed directly
 * (which only removes expansion error) and how sinks are grouped.
 *   out  nullable: the timings and the choice
 * Synchronises the stream; not allowed while capacities are reserved
 * (NBODY_ENOTSUP) or while a stream is being captured.
 */
typedef struct {
  int32_t ncand;           /* candidates timed */
  int32_t n_group[12];
  int32_t n_direct[12];
  double ms[12];           /* rebuild + forces, CUDA events */
  int32_t best;            /* index of the kept candidate */
} nbody_tune;
int nbody_autotune(nbody_tree *tree, nbody_tune *out, nbody_stream_t stream);

/* Read and clear the tree's device status word (blocks on the stream). */
int nbody_check(nbody_tree *tree, nbody_stream_t stream);
void nbody_tree_free(nbody_tree *tree);
const char *nbody_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */
