/*
 * cute.h -- C ABI of libcute_gb.so, GB300 (sm_103a) pair counting for
 * two-point correlation functions (Alonso 2012, "CUTE solutions for
 * two-point correlation functions from large cosmological datasets").
 *
 * The problem (Sec. 3.1 and Sec. 2.2, Eq. 11): given a data catalog D, a
 * random catalog R, separation bins and a separation measure, produce the
 * DD, DR and RR pair-count histograms and from them an estimator of the
 * correlation function (Eq. 13, 14, 15).  The separation measures are the
 * monopole distance, (sigma, pi) and (r, mu) (Sec. 2.1, Eq. 2-4) and the
 * angle between unit vectors (Eq. 7), binned on the squared chord.
 *
 * Conventions shared by every call:
 *   - Every call returns a cute_status; nothing aborts, exits or traps.  On
 *     failure the message is available from cute_last_error(ctx).
 *   - Pointers marked "host or device" may point to host memory (pageable
 *     or pinned) or to device memory of the context's device; the library
 *     detects which.  The caller keeps ownership of every pointer it passes.
 *   - Positions are FP64, row-major n x 3 (x0 y0 z0 x1 y1 z1 ...).
 *   - Auto-correlations (cat_a == cat_b) count each unordered pair i<j once;
 *     cross-correlations count every (i in A, j in B).  Histograms are
 *     uint64 per bin, row-major [axis0][axis1] for the 2-D kinds.
 *   - Bins are half-open, [e_b, e_{b+1}), compared on squared quantities
 *     (e_b * e_b in FP64).  Counts equal, bit for bit, those of the FP64
 *     canonical formulas below: pairs whose FP32 separation lies within a
 *     proven error bound of an edge are re-tested on the GPU (double-float
 *     with a carried error bound, then FP64 for pairs within it).
 *   - Work is enqueued on the context's CUDA stream.  Calls that write to
 *     host memory synchronise that stream before returning.
 */
#ifndef CUTE_H
#define CUTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cute_ctx cute_ctx; /* opaque; owns device memory and a stream */

typedef enum {
  CUTE_OK = 0,
  CUTE_E_INVALID = -1,     /* bad argument; nothing was enqueued          */
  CUTE_E_OOM = -2,         /* device or host allocation failed            */
  CUTE_E_CUDA = -3,        /* a CUDA runtime call failed                  */
  CUTE_E_STATE = -4,       /* object missing or in the wrong state        */
  CUTE_E_TIMEOUT = -5,     /* reserved: no kernel waits on another        */
  CUTE_E_UNSUPPORTED = -6, /* valid request the library does not implement */
  CUTE_E_DEVICE = -7       /* a kernel reported an internal inconsistency */
} cute_status;

/* Separation measure (Sec. 2.1). */
typedef enum {
  CUTE_MONO = 0,     /* |x_j - x_i|; edges0 = r edges                       */
  CUTE_R_MU = 1,     /* r and mu = |s.l|/(|s||l|), l = x_i + x_j (midpoint
                        line of sight, observer at the origin; open only);
                        edges0 = r edges, edges1 = mu edges, 0 ... 1         */
  CUTE_SIGMA_PI = 2, /* sigma = |(dx,dy)|, pi = |dz| (z line of sight);
                        edges0 = sigma edges, edges1 = pi edges             */
  CUTE_THETA = 3     /* chord |n_j - n_i| = 2 sin(theta/2) between unit
                        vectors (open only); edges0 = chord edges, see
                        cute_theta_to_chord                                  */
} cute_kind;

typedef enum {
  CUTE_PERIODIC = 0, /* cubic box [0, L)^3, minimum-image separations      */
  CUTE_OPEN = 1      /* no boundary (light cone, sky); no wrapping          */
} cute_boundary;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t of
   that device to enqueue on, or NULL for a stream the context creates and
   owns.  *out receives the context.  Errors: CUTE_E_INVALID (bad device or
   out == NULL), CUTE_E_CUDA, CUTE_E_OOM. */
cute_status cute_ctx_create(int device, void *cuda_stream, cute_ctx **out);

/* Wait for the context's work, free every catalog, plan and buffer it owns,
   and the context.  NULL is accepted and ignored. */
cute_status cute_ctx_destroy(cute_ctx *ctx);

/* Message of the last failed call on ctx (empty string if none).  The
   pointer stays valid until the next call on ctx.  ctx NULL -> a message
   about the last failed cute_ctx_create in this process. */
const char *cute_last_error(const cute_ctx *ctx);

/* Wait for all work enqueued on the context's stream and return the first
   deferred error a kernel reported (CUTE_E_DEVICE) or a CUDA error. */
cute_status cute_sync(cute_ctx *ctx);

/* ---------------------------------------------------------------- catalogs */

/* Copy a catalog to the device (Sec. 3.1: the x, y, z arrays of each
   catalog).  xyz: n x 3 FP64, host or device.  w: n FP32 weights (host or
   device) or NULL for unit weights.  Periodic catalogs must satisfy
   0 <= x < box_L on every axis, else CUTE_E_INVALID and no catalog is made.
   box_L is ignored for CUTE_OPEN.  The copy belongs to ctx until
   cute_catalog_free or cute_ctx_destroy.  *cat_id receives its handle.
   n may be 0.  n above 2^31 - 1 is CUTE_E_INVALID. */
cute_status cute_catalog_upload(cute_ctx *ctx, const double *xyz, const float *w,
                                int64_t n, cute_boundary boundary, double box_L,
                                int32_t *cat_id);

/* Free a catalog and its cell grid.  CUTE_E_STATE if cat_id is unknown. */
cute_status cute_catalog_free(cute_ctx *ctx, int32_t cat_id);

/* Number of objects of a catalog. */
cute_status cute_catalog_size(cute_ctx *ctx, int32_t cat_id, int64_t *n);

/* Cell grid (Sec. 3.3): cover the volume with cells no smaller than
   reach[k] / cells_per_reach on axis k and counting-sort every listed
   catalog into them, on ONE geometry shared by all of them (their joint
   bounding box for CUTE_OPEN, [0, L)^3 for CUTE_PERIODIC), so that any two
   of them can then be counted against each other.  reach[3] is the largest
   separation per axis that must be found (r_max on each axis for the
   monopole, (r,mu) and theta; (sigma_max, sigma_max, pi_max) for
   (sigma,pi)).  cells_per_reach: 1..8, or 0 to choose from the mean
   number of objects in a reach-sized box (below 600: 2, below 3000: 3,
   else 4).  Cells along x are 8 times finer (rows of cells run along x).
   The catalogs' joint extent must stay within 2e8 on every axis
   (CUTE_E_UNSUPPORTED otherwise: the kernels' padding sits at 1e9).
   All catalogs must have the same boundary (and box_L).  A periodic grid
   needs reach[k] <= 0.47 box_L, else CUTE_E_UNSUPPORTED.  Rebuilding a
   catalog's grid replaces the previous one. */
cute_status cute_grid_build(cute_ctx *ctx, const int32_t *cat_ids, int32_t n_cats,
                            const double reach[3], int32_t cells_per_reach);

/* ---------------------------------------------------------------- counting */

typedef struct {
  cute_kind kind;
  int32_t cat_a, cat_b;  /* cat_a == cat_b: auto-correlation (i<j)          */
  const double *edges0;  /* host; n0 + 1 strictly increasing values >= 0    */
  int32_t n0;
  const double *edges1;  /* host; n1 + 1 values for CUTE_R_MU (0 ... 1) and
                            CUTE_SIGMA_PI; NULL / 0 for the 1-D kinds       */
  int32_t n1;
  int32_t weighted;      /* 1: also produce sum of w_i w_j per bin (FP64)   */
} cute_pair_desc;

/* Count the pairs of d->cat_a x d->cat_b into bins (Sec. 2.2 Eq. 11; the
   hot loop of Sec. 3.1-3.2).  Both catalogs need cell grids of the same
   geometry whose reach covers the largest edge on every axis.
   counts: n0 * n1 (n1 = 1 for 1-D kinds) uint64, host or device.
   oor: if not NULL, receives the number of pairs that fall in no bin (all
        pairs of the pair set, N_A N_B or N (N - 1) / 2, minus the sum of
        counts); host.
   wsum: if d->weighted, n0 * n1 doubles (host or device) receiving the sum
        of w_i * w_j per bin, accurate to 1e-9 relative or better.
   Errors: CUTE_E_INVALID, CUTE_E_STATE (catalog or grid missing or on
   different geometries, reach too small), CUTE_E_UNSUPPORTED (kind not
   defined for the boundary; bins the error analysis cannot serve, e.g. a
   CUTE_R_MU count whose objects come closer to the observer than half the
   largest r edge, where the line of sight x_i + x_j can vanish), CUTE_E_CUDA,
   CUTE_E_DEVICE. */
cute_status cute_count_pairs(cute_ctx *ctx, const cute_pair_desc *d, uint64_t *counts,
                             uint64_t *oor, double *wsum);

/* Count n independent pair sets in ONE persistent launch (the many-mock
   use of Fig. 5).  All descriptors must share kind, edges and weighted.
   counts[k]: output of descriptor k as in cute_count_pairs (host or device).
   wsum may be NULL; else wsum[k] as in cute_count_pairs.  The result equals
   n separate cute_count_pairs calls bit for bit.  When every output is
   device memory, the call's work (counter resets, the kernel, the output
   copies) is captured once into a CUDA graph and replayed by later calls
   with the same descriptors and outputs. */
cute_status cute_count_pairs_batched(cute_ctx *ctx, int32_t n, const cute_pair_desc *d,
                                     uint64_t *const *counts, double *const *wsum);

/* Gradient of the weighted-count functional F = sum_b G_b W_b, W_b the
   weighted count of bin b (weights of Sec. 3.4), with respect to every
   object's weight:  dF/dw_i = sum_j w_j G[bin(i, j)] over i's partners
   (j != i for auto).  G: n0 * n1 doubles (host or device).  grad_a: n_a
   doubles, the gradient for catalog A's weights in A's upload order (host
   or device).  grad_b: for cross counts, n_b doubles for catalog B's
   weights (host or device), or NULL to skip; ignored for auto. */
cute_status cute_count_pairs_adjoint(cute_ctx *ctx, const cute_pair_desc *d, const double *G,
                                     double *grad_a, double *grad_b);

/* Counts like cute_count_pairs, but allocates no device memory: for callers
   that cannot let a library call cudaMalloc when they count -- a framework
   whose caching allocator owns the device memory (a stray cudaMalloc
   fragments its pool or fails once the pool has taken the device), or loops
   where cudaMalloc and cudaFree would synchronise the device.  The paper has
   no counterpart; it is a deployment form of the counting kernel.
   The catalogs and grids must already exist (upload and grid build allocate
   and are done beforehand).  counts (n0 * n1 uint64) and, if d->weighted,
   wsum (n0 * n1 doubles) must be device memory of the context's device;
   host pointers are CUTE_E_INVALID.  The kernel's scratch (work items,
   binning tables, work counters) lives in one fixed 8 MiB device array of
   the library, held on every device that loads it until the process exits;
   a request whose scratch exceeds 8 MiB is rejected with CUTE_E_INVALID and
   a message naming the size (count smaller catalogs, or use
   cute_count_pairs).  The first call on a device looks up the array's
   device address (cudaGetSymbolAddress) with that device current.  Each
   call builds its work-item records on the host (its host time grows with
   the number of items) and copies them, with the binning tables, from
   pageable host memory: that copy waits for the context's stream.  Every
   call shares the array and leaves its
   contents behind (the counters are cleared at the start of each call):
   calls that overlap on the GPU -- on different streams or contexts -- race
   on it.  Asynchronous on the context's stream; cute_sync reports kernel
   errors.  cute_last_stats does not describe these calls. */
cute_status cute_count_pairs_noalloc(cute_ctx *ctx, const cute_pair_desc *d, uint64_t *counts,
                                     double *wsum);

/* Statistics of the last count call on ctx. */
typedef struct {
  uint64_t candidate_pairs; /* pairs examined by the FP32 path (after the
                               neighbour cull; see stencil_pairs)           */
  uint64_t rechecked_pairs; /* of those, re-tested near an edge            */
  uint64_t fp64_pairs;      /* of those, decided by the FP64 formula (the
                               double-float stage left them open)          */
  uint64_t pair_slots;      /* (home, neighbour) slots the kernel evaluated,
                               including empty and padding slots            */
  uint64_t work_items;      /* (home chunk, neighbour slice) items run      */
  int32_t launches;         /* kernels launched by the call                 */
  int32_t warps_per_block, blocks, home_per_lane;
  float kernel_ms;          /* device time of the counting kernel(s), if
                               timing was enabled with cute_set_timing     */
  uint64_t stencil_pairs;   /* pairs the cell stencil presented (Sec. 3.3),
                               before the kernel dropped the neighbours
                               beyond the reach of a home chunk's bounding
                               box: candidate_pairs <= stencil_pairs        */
} cute_stats;
cute_status cute_last_stats(cute_ctx *ctx, cute_stats *out);

/* Enable (1) or disable (0) CUDA-event timing of the counting kernels
   (adds two events per call; off by default). */
cute_status cute_set_timing(cute_ctx *ctx, int32_t on);

/* Launch shape override for the counting kernel: home_per_lane in {2, 4}
   (objects of A held per lane; 0 = library default), warps_per_block
   (0 = library default: the most the kernel allows; at most 20 for plain
   monopole and theta counts with 2 home objects per lane, 16 otherwise;
   fewer if shared memory requires), slice (neighbour objects per work item, 0 = default, multiple
   of 64).  table_binning = 1 bins through lookup tables
   even when the edges are uniform (0 = arithmetic binning for uniform
   edges).  Used by the autotuner and by tests of both binning paths. */
cute_status cute_set_launch(cute_ctx *ctx, int32_t home_per_lane, int32_t warps_per_block,
                            int32_t slice, int32_t table_binning);

/* Autotuner: picks the launch shape of the counting kernel for the given
   descriptors (all sharing kind, edges and weighting) by timing candidates
   on the GPU -- home objects per lane {2, 4}, warps per block {8, 12, 16,
   20 where the kernel allows it}
   (within shared memory), neighbour slice {1024, 2048, 4096} -- each on at
   most max_items work items; if tune_cells, it also rebuilds the grids of
   the descriptors' catalogs at 2, 3 and 4 cells per reach and keeps the
   fastest.  The choice is remembered for these catalogs and used by later
   counts (cute_set_launch overrides it).  *out (may be NULL) receives it. */
typedef struct {
  int32_t cells_per_reach, home_per_lane, warps_per_block, slice;
  float ms; /* time of the chosen shape on the timed items */
} cute_tuning;
cute_status cute_autotune(cute_ctx *ctx, int32_t n, const cute_pair_desc *d, int32_t tune_cells,
                          int64_t max_items, cute_tuning *out);

/* ---------------------------------------------------------------- estimators
   Host FP64 arithmetic on exact counts (Sec. 2.2).  Counts are unique pairs.
   A bin whose denominator is zero gives NaN.  No device work, no context. */
typedef enum {
  CUTE_EST_PERIODIC = 0, /* Eq. 13 with N(N-1)/2 pairs and exact shells:
                            xi = DD / (N(N-1)/2 * 4pi/3 (e1^3 - e0^3) / L^3) - 1;
                            uses DD, Nd, edges, box_L                        */
  CUTE_EST_NATURAL = 1,  /* Eq. 14: Nr(Nr-1)/(Nd(Nd-1)) DD/RR - 1          */
  CUTE_EST_LS = 2        /* Eq. 15: (Nr(Nr-1)/(Nd(Nd-1)) DD - (Nr-1)/Nd DR
                            + RR) / RR                                       */
} cute_estimator_kind;

/* DD, DR, RR: nbins uint64 on the host (DR/RR may be NULL when unused);
   edges: nbins + 1 r edges (periodic only); xi_out: nbins doubles, host. */
cute_status cute_estimator(cute_estimator_kind k, const uint64_t *DD, const uint64_t *DR,
                           const uint64_t *RR, int64_t Nd, int64_t Nr, int32_t nbins,
                           const double *edges, double box_L, double *xi_out);

/* Chord between unit vectors an angle theta apart (Eq. 7 gives
   cos theta = n_1 . n_2): chord = 2 sin(theta/2), theta in degrees, FP64,
   host.  The chord is monotone in theta, so binning chords on these edges
   bins theta on the given angles. */
cute_status cute_theta_to_chord(const double *theta_deg, int32_t n, double *chord_out);

/* ---------------------------------------------------------------- sky input */

/* Background cosmology for comoving distances: present-day matter and
   dark-energy densities (curvature 1 - omega_m - omega_l) and a constant
   dark-energy equation of state w0 (-1: a cosmological constant). */
typedef struct {
  double omega_m, omega_l, w0;
} cute_cosmology;

/* Positions from sky coordinates, on the GPU.  ra, dec: n angles in
   degrees; z: n redshifts in [0, 20], or NULL for unit vectors (the
   projection onto the unit sphere of Sec. 3.4.2, for CUTE_THETA).  xyz: n x 3
   doubles, row-major, = chi(z) (cos dec cos ra, cos dec sin ra, sin dec) in
   Mpc/h, chi(z) = (c/H0) integral_0^z dz'/E(z') the radial comoving
   distance of Sec. 2.1, c/H0 = 2997.92458 Mpc/h, E(z)^2 = omega_m (1+z)^3 +
   (1 - omega_m - omega_l) (1+z)^2 + omega_l (1+z)^(3 (1 + w0)); positions
   are placed along n at that distance (the flat-space separations of
   Eq. 9).  chi is interpolated from an FP64 table (relative error below
   1e-12).  All four arrays on the device of ctx, or all on the host; the
   call returns when xyz is written.  Errors: CUTE_E_INVALID (null
   pointers, n < 0, z without cosmology, E(z) <= 0 below z = 20, a redshift
   outside [0, 20] or NaN), CUTE_E_OOM, CUTE_E_CUDA. */
cute_status cute_sky_to_xyz(cute_ctx *ctx, const double *ra, const double *dec, const double *z,
                            int64_t n, const cute_cosmology *cosmo, double *xyz);

/* ---------------------------------------------------------------- pixel maps */

/* Pixel map of an angular catalog (Sec. 3.4.2: correlate pixels weighted by
   the objects they hold instead of the objects), on the GPU.  Pixelisation:
   HEALPix RING (12 nside^2 equal-area pixels; the paper leaves the scheme
   open).  xyz: n x 3 unit vectors (|x|^2 within 1e-6 of 1, else
   CUTE_E_INVALID); w: n object weights or NULL for 1; map: 12 nside^2
   doubles, overwritten with the summed weight of every pixel.  nside: a power
   of 2 up to 8192.  All arrays on the device of ctx, or all on the host;
   returns when map is written.  Pixel weights become FP32 catalog weights
   when the pixels are uploaded (exact for integer counts below 2^24). */
cute_status cute_pixel_map(cute_ctx *ctx, const double *xyz, const float *w, int64_t n,
                           int32_t nside, double *map);

/* Centres of HEALPix RING pixels pix[0..m) as unit vectors xyz (m x 3), on
   the GPU; arrays both on the device or both on the host.  CUTE_E_INVALID
   for an index outside 0 .. 12 nside^2 - 1. */
cute_status cute_pixel_centres(cute_ctx *ctx, int32_t nside, const int64_t *pix, int64_t m,
                               double *xyz);

/* Estimators on weighted pair sums (pixel maps, weighted catalogs): Eq. 14
   (CUTE_EST_NATURAL) or Eq. 15 (CUTE_EST_LS) with every count divided by its
   total pair weight: DD by (S_d^2 - Q_d) / 2, DR by S_d S_r, RR by
   (S_r^2 - Q_r) / 2, where S and Q are the sums of the weights and of their
   squares (unit weights give the unique-pair normalisation of
   cute_estimator).  DD, DR (LS only), RR: nbins doubles, host.  NaN where
   RR = 0.  Errors: CUTE_E_INVALID (null pointers, nbins < 1, a non-positive
   total pair weight, CUTE_EST_PERIODIC). */
cute_status cute_estimator_weighted(cute_estimator_kind k, const double *DD, const double *DR,
                                    const double *RR, double s_d, double q_d, double s_r,
                                    double q_r, int32_t nbins, double *xi_out);

/* ---------------------------------------------------------------- density grid */

/* Monopole of a periodic box from a density grid (Sec. 3.4.4), on the GPU:
   the objects (xyz: n_obj x 3 in [0, box_L), w: weights or NULL for 1) are
   interpolated to an ngrid^3 grid (grid points at multiples of
   a = box_L / ngrid) with the triangular-shaped-cloud kernel, the
   overdensity delta = rho / mean(rho) - 1 is formed, and xi_b is the mean of
   delta_i delta_j over the pairs of distinct grid points whose separation r
   (periodic, squared in FP64) falls in [e_b, e_b+1).  ngrid: a multiple of
   32 in 32..1024; r_max = edges[nbins] below box_L / 2 and at least a.
   xi_out: nbins doubles (NaN for a bin no lag falls in); lags_out (or NULL):
   the number of lag vectors per bin (each unordered pair direction once).
   xyz and w both on the device of ctx or both on the host; outputs on the
   host; returns when done.  Results are FP32 lag sums with float-float
   accumulation: relative error about 1e-6 of the sum of |delta_i delta_j|.
   Errors: CUTE_E_INVALID (arguments, positions outside the box, total weight
   <= 0), CUTE_E_OOM, CUTE_E_CUDA. */
cute_status cute_density_grid_xi(cute_ctx *ctx, const double *xyz, const float *w, int64_t n_obj,
                                 double box_L, int32_t ngrid, const double *edges, int32_t nbins,
                                 double *xi_out, double *lags_out);

/* Multipoles of xi(r, mu) (Eq. 3: xi(r, mu) = sum_l xi_l(r) P_l(mu), whose
   l = 0 term is the monopole of Eq. 4).  With mu = |cos| in [0, 1] the even
   multipoles are xi_l(r) = (2l + 1) * integral_0^1 xi(r, mu) P_l(mu) dmu,
   and xi is taken constant within each mu bin, so bin k contributes
   xi(r, k) * [P_{l+1} - P_{l-1}] from m_k to m_{k+1} (l >= 1; for l = 0 the
   bin width).  xi: n_r x n_mu doubles, row-major [r][mu] (as
   cute_count_pairs and cute_estimator give them); mu_edges: n_mu + 1
   increasing values from 0 to 1; ells: n_ell even multipole orders in
   0..16; out: n_ell x n_r doubles, [ell][r].  A NaN bin makes that r's
   multipoles NaN.  FP64, host.  Errors: CUTE_E_INVALID (null pointers,
   sizes < 1, edges not covering [0, 1] in increasing order, odd or out of
   range orders). */
cute_status cute_multipoles(const double *xi, int32_t n_r, int32_t n_mu, const double *mu_edges,
                            int32_t n_ell, const int32_t *ells, double *out);

/* Library version string. */
const char *cute_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CUTE_H */
