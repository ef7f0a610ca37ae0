/* ww.h — C-ABI of the B300 Whirlwind MCF phase-unwrapping library (libww.so).
 *
 * The library implements the hot path of the minimum-cost-flow (MCF) 2D phase
 * unwrapper of Staniewicz et al., "A Probabilistic-Cost Algorithm for
 * Large-Scale 2D Phase Unwrapping" (arxiv 2609.36267), Sec. II:
 *   1. residues of the wrapped phase (Sec. II-A, Eq. 1),
 *   2. integer likelihood-ratio arc costs from a compact lookup table
 *      (Sec. II-B, Eqs. 4-7),
 *   3. the MCF solve (Sec. II-A Eq. 2) by successive shortest paths with node
 *      potentials and one augmentation per shortest-path tree (Sec. II-C),
 *   4. integration of the flows into integer cycle counts (Sec. II-A, II-C).
 * Every step runs as CUDA kernels on the caller's stream; no torch types appear
 * here and the library never falls back to the CPU.
 *
 * Array conventions (all row-major, m rows x n columns of pixels, m,n >= 2):
 *   Pixel edge h(i,j) joins (i,j)->(i,j+1); v(i,j) joins (i,j)->(i+1,j).  Edge
 *   arrays are m x n planes (the unused last column of h / last row of v is
 *   written as 0).
 *   Dual node p=(i,j), 0<=i<m-1, 0<=j<n-1, is the 2x2 loop whose top-left pixel
 *   is (i,j); node arrays hold (m-1)*(n-1) entries, index i*(n-1)+j.  The ground
 *   node G (the image's outer ring, Sec. II-A, collapsed into one node) follows
 *   as index (m-1)*(n-1) where a node array carries it.
 *   h(i,j) separates node (i-1,j) [above] from (i,j) [below]; v(i,j) separates
 *   node (i,j-1) [left] from (i,j) [right]; neighbours outside the grid are G.
 *   Costs: int16 planes [4][m][n]: 0 = arc above->below across h (adds +1 to the
 *   cycle difference dk_h), 1 = below->above (dk_h -1), 2 = right->left across v
 *   (dk_v +1), 3 = left->right (dk_v -1).
 *   Flows: int8 planes [2][m][n] holding dk_h, dk_v in {-1,0,1}.
 *   Wrap count n_e = [dpsi > PI_F] - [dpsi <= -PI_F] for dpsi = psi_v - psi_u in
 *   fp32 (PI_F = fp32 nearest pi); the residue of node (i,j) is
 *   r = -(n_h(i,j) + n_v(i,j+1) - n_h(i+1,j) - n_v(i,j)) and r_G = -sum(r).
 *   Cycle counts: K(0,0)=0, K_v = K_u + dk_e - n_e; unwrapped
 *   phi = (float)((double)psi + (double)K * 2pi), NaN at invalid pixels.
 *
 * Input validity: a pixel is valid iff mask != 0 (mask may be NULL = all valid)
 * and its phase (or both complex parts) and coherence are finite.  Invalid
 * pixels are treated as phase 0, coherence 0; arcs of edges touching them cost
 * 0 (Sec. II-B).  A complex64 input (interleaved re, im) is converted to phase
 * by the library's own fixed-point CORDIC atan2 (30 iterations, angle unit
 * 2^-29 rad), identical on every device.
 *
 * Pointers: unless stated, array arguments are DEVICE pointers owned by the
 * caller, and calls are asynchronous on `stream` (0 = legacy default stream).
 * Host-side argument checks return a status immediately; device-side failures
 * of the solver are written to its device status word.
 */
#ifndef WW_H
#define WW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ww_status;
#define WW_OK 0
#define WW_ERR_INVALID_ARG (-1)   /* bad pointer, size or parameter */
#define WW_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define WW_ERR_OOM (-3)           /* device or host allocation failed */
#define WW_ERR_INFEASIBLE (-4)    /* supplies cannot be routed with unit capacities */
#define WW_ERR_TIMEOUT (-5)       /* a bounded device loop hit its limit; state resumable */
#define WW_ERR_OVERFLOW (-6)      /* a 32-bit distance or reduced cost overflowed */
#define WW_ERR_NOT_IMPLEMENTED (-7)
#define WW_ERR_INTERNAL (-8)      /* an invariant check failed (e.g. negative reduced cost) */

typedef void* ww_stream;  /* a cudaStream_t */

/* Human-readable name of a status code (static string). */
const char* ww_status_string(ww_status s);

/* Parameters.  ww_params_default fills the paper's values (Sec. II-B, II-C). */
typedef struct ww_params {
  int32_t box_half_width;   /* slope-estimate window half width; 2 = 5x5 (Sec. II-B) */
  float steep_rad;          /* unsmoothed |gradient| above which an edge costs 0: 1.0 (Sec. II-B) */
  int32_t steep_cap_ppm;    /* cap on zeroed steep edges, per million valid edges: 30000 = 3% */
  int32_t max_passes;       /* solver pass limit -> WW_ERR_TIMEOUT (default 100000) */
  int32_t wait_polls;       /* polls (~0.1-0.2 us each) of any device worklist wait before it gives
                               up: the search then stops, the pass augments nothing and the solve
                               returns WW_ERR_TIMEOUT with flows and potentials of the last complete
                               pass (resumable, see ww_solve_mcf_resume); default 2^25, >= 1 */
  int32_t graph_loop;       /* 1 = the pass loop runs on the device inside one CUDA graph launch
                               (conditional while node; default), 0 = one host sync per pass */
  /* search schedule: the optimum does not depend on it (ww_autotune_batch picks it).
   * A banded pass searches only up to a distance cap; if no imbalanced node is
   * reached below the cap, the cap widens (x band_growth, at most three times,
   * the last time to no cap) and the search resumes from the tiles that were cut. */
  int32_t search_ctas_per_sm; /* persistent search CTAs per SM, 0 = as many as fit (default) */
  int32_t band_min;         /* smallest cap of a banded pass (default 1024), >= 1 */
  int32_t band_mult;        /* cap = max(band_min, band_mult x the last augmented distance) (4) */
  int32_t band_growth;      /* cap widening factor, 2..64 (8) */
  int32_t band_start_ppm;   /* passes are banded once fewer than this many per million nodes are
                               imbalanced (default 1000000 = always) */
  int32_t full_passes;      /* the first passes search without a cap (default 0) */
  int32_t ground_sink_below; /* while at most this many nodes are imbalanced, the ground is no
                               root of the search but a sink reached through the border arcs
                               (a pass then augments only up to the ground's distance); 0 = never */
  int32_t zero_stop_below;  /* while at most this many nodes are imbalanced, a banded pass first
                               searches at distance 0 only, within zero_band_hops hops of the
                               roots, and augments there if it reaches an imbalanced node
                               (zero-cost paths, no potential change); default 64; 0 = never */
  int32_t zero_band_hops;   /* largest hop radius of that first band (default 512) */
  int32_t zero_band_hops_min; /* its first hop radius (default 512 = one stage): below
                               zero_band_hops the band is searched with radius min, then
                               sqrt(min * max), then max hops, widening only while no
                               imbalanced node is reached (each stage a fixed point) */
  /* cost-model variants (Sec. II-B leaves both choices open); every step stays
   * bit-reproducible (integer or singly rounded fp32 operations only) */
  int32_t slope_estimator;  /* 0 = fixed-point mean of the wrapped gradients in the window
                               (default); 1 = argument of the sum of their unit phasors
                               exp(i d), each from a fixed-point CORDIC rotation of
                               round(d 2^29) (length 2^30), summed as integers, the argument
                               by the CORDIC atan2 of the two sums each rounded once to fp32 */
  int32_t cost_lookup;      /* 0 = nearest bin of the int16 table (default); 1 = bilinear
                               interpolation, between bin centres, of the table's FP64
                               100 ln(P0/P+) kept in fp32 (x = (a + PI_F) fp32(256/2pi) - 1/2,
                               y = g 128 - 1/2, outermost pair and weights clamped,
                               v0 = r00 + fx (r01 - r00), v1 likewise, v = v0 + fy (v1 - v0)),
                               then floor, saturated to [0, 32767] */
} ww_params;
void ww_params_default(ww_params* p);

/* ---- Cost lookup table (Sec. II-B, Eqs. 4-7) ----
 * A table holds floor(100 c) as int16 (saturated at 32767) for c of Eq. 4 on a
 * 128 (coherence) x 256 (slope) grid of bin centres gamma_k = (k+1/2)/128,
 * alpha_j = -pi + (j+1/2) 2pi/256, for one number of looks L.  Edge lookup:
 * j = clamp(floor((a + PI_F) * fp32(256/2pi)), 0, 255),
 * k = clamp(floor(gamma_e * 128), 0, 127) in fp32 with no fused operations,
 * gamma_e = min of the endpoint coherences, a = box-filtered slope estimate. */
typedef struct ww_lut ww_lut;

/* Build the table in FP64 on the host (coherence-marginalised L-look phase
 * noise, Eq. 5; edge-noise convolution; Eq. 6 tail probabilities; Gaussian
 * slope marginalisation over +-8 sigma, Eq. 7).  nlooks must be > 1.  Takes a
 * few seconds of host time; the result is cached per nlooks inside the library
 * and the returned handle shares it.  *out is owned by the caller (ww_lut_free). */
ww_status ww_build_lut(double nlooks, ww_lut** out);
/* Wrap a caller-supplied host table (128*256 int16, row = coherence bin). */
ww_status ww_lut_from_table(double nlooks, const int16_t* host_table, ww_lut** out);
/* The same with the fp32 table of 100 ln(P0/P+) (128*256) that the
 * interpolated lookup (ww_params.cost_lookup = 1) reads. */
ww_status ww_lut_from_tables(double nlooks, const int16_t* host_table, const float* ratio100, ww_lut** out);
/* Copy out that fp32 table (built tables and ww_lut_from_tables only). */
ww_status ww_lut_ratio_table(const ww_lut* lut, float* ratio100);
/* Copy out the host table (128*256) and, for built tables, 100*c in FP64
 * before flooring (cost100 may be NULL). */
ww_status ww_lut_table(const ww_lut* lut, int16_t* host_table, double* cost100);
void ww_lut_free(ww_lut* lut);

/* ---- Workspace: library-owned device scratch for one request at a time ----
 * Sized for grids up to max_rows x max_cols; allocated with cudaMalloc on the
 * current device.  One workspace must not be used by two calls that overlap
 * on the GPU. */
typedef struct ww_workspace ww_workspace;
ww_status ww_workspace_create(int64_t max_rows, int64_t max_cols, ww_workspace** out);
void ww_workspace_free(ww_workspace* ws);
/* Bytes of device memory a workspace for m x n takes. */
int64_t ww_workspace_bytes(int64_t m, int64_t n);

/* ---- Step 1: residues (Sec. II-A, Eq. 1) ----
 * ifg: float32 phase [m][n] (is_complex=0) or interleaved complex64 [m][n][2]
 * (is_complex=1).  coh (may be NULL) and mask (may be NULL) only decide
 * validity here.  residues: int8 [(m-1)(n-1)]; ground: device int32[1], r_G. */
ww_status ww_residues(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                      int64_t m, int64_t n, int8_t* residues, int32_t* ground, ww_stream stream);

/* ---- Step 2: arc costs (Sec. II-B) ----
 * Writes costs [4][m][n] int16 as described above, including the steep-edge
 * bound (at most steep_cap_ppm of valid edges with |d| > steep_rad get cost 0,
 * largest |d| first, ties by edge index with h before v).  ws provides scratch
 * for the steep selection. */
ww_status ww_costs(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                   int64_t m, int64_t n, const ww_lut* lut, const ww_params* params,
                   ww_workspace* ws, int16_t* costs, ww_stream stream);

/* Same output as ww_costs, for callers that cannot allocate device memory: for
 * example code whose device memory is owned by another allocator (a
 * framework's caching pool) or a real-time loop that must not pay cudaMalloc's
 * implicit device synchronisation.  The paper has no counterpart; this is an
 * interface variant.  It calls no cudaMalloc/cudaFree and takes no workspace:
 * the steep-edge selection scratch and a copy of the cost table live in one
 * file-scope device array of about 1.4 MB that every GPU loading the library
 * holds until the process exits.  Limit: m*n <= 2^27 pixels (134,217,728);
 * larger grids return WW_ERR_INVALID_ARG, and so do parameters ww_costs would
 * refuse and the cost-model variants (slope_estimator, cost_lookup other than 0).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every later call enqueues only an upload of the
 * table from a page-locked host copy made when the table was built, two
 * memsets and kernel launches, so it neither waits for the stream nor
 * prevents capturing the call into a CUDA graph (if the page-locked copy
 * could not be made, the upload comes from pageable memory, which does both).
 * All calls share the array and each rewrites it (table copy, cleared
 * counters), so calls that overlap on the GPU race and must be serialised by
 * the caller (e.g. one stream). */
ww_status ww_costs_noalloc(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                           int64_t m, int64_t n, const ww_lut* lut, const ww_params* params,
                           int16_t* costs, ww_stream stream);

/* ---- Step 3: MCF solve (Sec. II-A Eq. 2, Sec. II-C) ----
 * Exact successive-shortest-path solve of Eq. 2 with unit capacities.
 * Outputs: flows [2][m][n] (dk in {-1,0,1}), potentials int64 [(m-1)(n-1)+1]
 * (the last entry is G) certifying optimality: every residual arc has reduced
 * cost c - p(tail) + p(head) >= 0; total_cost: device int64[1] = sum c_a x_a;
 * dev_status: device int32[1] (WW_OK, WW_ERR_INFEASIBLE, WW_ERR_TIMEOUT,
 * WW_ERR_OVERFLOW, WW_ERR_INTERNAL).  The pass loop runs on the device inside
 * one CUDA graph launch (params->graph_loop = 1, the default) or is driven by
 * the host with one stream synchronisation per pass (graph_loop = 0); either
 * way the call returns when the solve has finished (the stream is
 * synchronised) and the returned status equals *dev_status.  On
 * WW_ERR_TIMEOUT (pass limit or worklist wait limit) flows and potentials hold
 * the state after the last complete pass: every residual arc has a
 * non-negative reduced cost, and ww_solve_mcf_resume continues from it. */
ww_status ww_solve_mcf(const int8_t* residues, const int32_t* ground, const int16_t* costs,
                       int64_t m, int64_t n, const ww_params* params, ww_workspace* ws,
                       int8_t* flows, int64_t* potentials, int64_t* total_cost,
                       int32_t* dev_status, ww_stream stream);

/* Continue a solve from given flows and potentials (checkpoint/resume; the
 * paper's solver has no counterpart).  flows (IN/OUT, [2][m][n], |dk| <= 1)
 * and potentials (IN/OUT, (m-1)(n-1)+1, ground last) are typically what an
 * earlier ww_solve_mcf or ww_solve_mcf_resume returned with WW_ERR_TIMEOUT, or
 * a copy of them saved to host memory and loaded back.  Any pair in which
 * every residual arc has a non-negative reduced cost (c - p(tail) + p(head) >= 0)
 * is accepted: the imbalance left by the flows is then routed by successive
 * shortest paths exactly as in ww_solve_mcf, so the result is an optimum of
 * Eq. 2 with its certificate.  The pair is checked on the device first; a pair
 * with |dk| > 1, flow on a missing edge or a negative reduced cost returns
 * WW_ERR_INVALID_ARG without changing it.  Synchronises the stream. */
ww_status ww_solve_mcf_resume(const int8_t* residues, const int32_t* ground, const int16_t* costs,
                              int64_t m, int64_t n, const ww_params* params, ww_workspace* ws,
                              int8_t* flows, int64_t* potentials, int64_t* total_cost,
                              int32_t* dev_status, ww_stream stream);

/* Solver statistics of the last solve (ww_solve_mcf, ww_solve_mcf_resume or
 * ww_unwrap) on this workspace (host struct). */
typedef struct ww_solve_stats {
  int64_t passes, augmentations, search_iterations, tile_visits;
  int64_t residues, ground_net;
  double ms_search;      /* host wall time of the pass loop (searches, selection, augmentation, potentials) */
  double ms_other;       /* host wall time of the rest of the solve (session setup, finalisation) */
  double ms_search_gpu;  /* device time of the search launches (CUDA events; host-driven pass loop only, 0 with graph_loop) */
  int64_t local_rounds;  /* local fixed-point rounds (four concurrent line sweeps each) summed over tile visits */
  int64_t visit_cycles;  /* SM clock cycles summed over tile visits */
  int64_t load_cycles;   /* of which: loading labels and computing reduced arc costs */
  int64_t relax_cycles;  /* of which: the local fixed point (line sweeps) */
  int64_t settled_visits; /* nodes reached (finite label) at the end of a tile visit, summed over visits */
  int64_t narrow_visits;  /* tile visits relaxed in 32-bit keys (label spans small enough) */
  int64_t narrow_redone;  /* of which redone in 64-bit keys (a candidate left the 32-bit range) */
} ww_solve_stats;
ww_status ww_get_solve_stats(const ww_workspace* ws, ww_solve_stats* out);

/* ---- Step 4: integration (Sec. II-A, II-C) ----
 * unwrapped: float32 [m][n]; cycles: int32 [m][n]. */
ww_status ww_integrate(const void* ifg, int32_t is_complex, const float* coh, const uint8_t* mask,
                       const int8_t* flows, int64_t m, int64_t n, float* unwrapped, int32_t* cycles,
                       ww_stream stream);

/* ---- Whole path ----
 * Residues, costs (table for nlooks, cached), MCF, integration.  total_cost is
 * a HOST int64* (may be NULL).  Synchronises the stream; returns the solver's
 * status.  Scratch for residues, costs, flows and potentials comes from ws. */
ww_status ww_unwrap(const void* ifg, int32_t is_complex, const float* coh, double nlooks,
                    const uint8_t* mask, int64_t m, int64_t n, const ww_params* params,
                    ww_workspace* ws, float* unwrapped, int32_t* cycles, int64_t* total_cost,
                    ww_stream stream);

/* Device arrays the last ww_unwrap on this workspace solved and certified
 * with: residues ((m-1)(n-1)), ground charge (1), cost planes ([4][m][n]),
 * flows ([2][m][n]) and potentials ((m-1)(n-1)+1), laid out for that call's
 * m x n.  They are workspace memory: valid until the next call that uses the
 * workspace, not to be freed.  Any output pointer may be NULL. */
ww_status ww_workspace_last_unwrap(const ww_workspace* ws, const int8_t** residues, const int32_t** ground,
                                   const int16_t** costs, const int8_t** flows, const int64_t** potentials);

/* ---- Connected-component labels (Sec. II-D) ----
 * After unwrapping, a pixel edge is reliable when both of its pixels are
 * valid and moving its ambiguity difference dk by +1 or by -1 would raise the
 * MCF objective by more than `threshold` (cost units of the int16 planes).
 * With unit capacities that is: dk = 0 on the edge and min(c+, c-) >
 * threshold (an edge that carries flow can drop it at a negative change).
 * Labels grow over reliable edges (4-neighbour components).
 *   costs: DEVICE int16 [4][m][n] as written by ww_costs; flows: DEVICE int8
 *   [2][m][n] as written by ww_solve_mcf (plane 0: dk of the edge
 *   (i,j)-(i,j+1) with costs planes 0/1 for +1/-1; plane 1: dk of
 *   (i,j)-(i+1,j) with planes 2/3); unwrapped: DEVICE float32 [m][n], NaN
 *   where invalid (as written by ww_integrate / ww_unwrap).
 *   labels: DEVICE int32 [m][n], caller-owned: 1 + the smallest row-major
 *   index of the pixel's component, 0 where invalid; unique whatever the
 *   schedule.  Also the union-find scratch: nothing is allocated.
 * Needs 1 <= m, n and m*n < 2^31, threshold >= 0 (else WW_ERR_INVALID_ARG).
 * Asynchronous on the stream; every device loop is bounded by the pixel count. */
ww_status ww_components(const int16_t* costs, const int8_t* flows, const float* unwrapped, int64_t m,
                        int64_t n, int32_t threshold, int32_t* labels, ww_stream stream);

/* ---- Bridging of mask-separated regions (Sec. II-D) ----
 * A mask that separates the valid pixels into several 4-connected regions
 * leaves their relative 2pi levels undetermined.  The regions are taken in
 * order of decreasing size (ties: smaller first row-major pixel); each region
 * after the first attaches to the nearest region already taken through the
 * closest pair of pixels (squared Euclidean distance; ties: the earlier parent
 * region, then the smaller parent pixel index, then the smaller child pixel
 * index).  Across each such edge the offset is
 * rint((median_parent - median_child) / 2pi) cycles (half to even), each
 * median taken in FP64 over the unwrapped phase of the endpoint's own region
 * inside a window x window box centred on the endpoint (the middle value, or
 * the mean of the two middle values), with the parent's offset already
 * applied, so offsets propagate from parent to child.  The paper uses 65-pixel
 * windows.
 *   unwrapped: DEVICE float32 [m][n], IN/OUT, NaN where invalid (as ww_unwrap
 *     writes it); valid pixels become (float)((double)phi + 2pi * offset).
 *   cycles: DEVICE int32 [m][n] or NULL, IN/OUT: offset added to each valid pixel.
 *   region: DEVICE int32 [m][n] or NULL, OUT: the pixel's region rank (0 =
 *     largest), -1 where invalid.  shift: DEVICE int32 [m][n] or NULL, OUT: the
 *     offset applied (0 where invalid).  n_regions: HOST int32 or NULL.
 * window: odd, 1..127.  Needs m*n < 2^31.  Allocates its scratch (about 16
 * bytes per pixel) with cudaMalloc and frees it before returning; synchronises
 * the stream (the size order of the regions is sorted on the host). */
ww_status ww_bridge(float* unwrapped, int32_t* cycles, int64_t m, int64_t n, int32_t window, int32_t* region,
                    int32_t* shift, int32_t* n_regions, ww_stream stream);

/* ---- Preprocessing: multilook and Eq. (3) sample coherence ----
 * From two co-registered SLC images slc1, slc2 (DEVICE interleaved complex64
 * [M][N]) over looks_y x looks_x looks: the multilooked interferogram
 * ifg = sum z1 conj(z2) (DEVICE complex64 [M/looks_y][N/looks_x], trailing
 * rows and columns that do not fill a window dropped) and the sample coherence
 * of Eq. 3, coh = |sum z1 conj(z2)| / sqrt(sum |z1|^2 sum |z2|^2) (DEVICE float32,
 * clamped to 1, 0 where a power sum is 0).  The looks are summed row-major in
 * fp32, every product and sum rounded once in the order
 *   t = (re1 re2 + im1 im2, im1 re2 - re1 im2), S12 += t, S11 += re1^2 + im1^2, ...
 * so the result is the same on every device.  Asynchronous. */
ww_status ww_multilook(const void* slc1, const void* slc2, int64_t M, int64_t N, int32_t looks_y, int32_t looks_x,
                       void* ifg, float* coh, ww_stream stream);

/* ---- Preprocessing: adaptive power-spectrum (Goldstein) filter (Sec. II-D) ----
 * ifg: DEVICE complex64 [m][n]; out: DEVICE complex64 [m][n] (not ifg).
 * Patches of 32 x 32 pixels start at every multiple of `step` (1..32) inside the
 * image (pixels beyond it count as 0).  Per patch: Z = DFT(patch); S = the
 * smooth x smooth (odd) circular box mean of |Z| divided by its maximum;
 * Z' = Z S^alpha (alpha >= 0); inverse DFT; the patches are added with the
 * separable weight w(t) = 1 - |(2t+1)/32 - 1| and the sum divided by the
 * summed weights.  fp32 arithmetic (agrees with an FP64 evaluation to about
 * 1e-5 of the local amplitude).  Allocates patch scratch (8 KB per patch) with
 * cudaMalloc and synchronises the stream before freeing it. */
ww_status ww_goldstein(const void* ifg, int64_t m, int64_t n, float alpha, int32_t step, int32_t smooth, void* out,
                       ww_stream stream);

/* ---- Cycle transfer after preprocessing (Sec. II-D) ----
 * The unwrapped phase of a filtered interferogram fixes the integer cycles of
 * the original wrapped phase: K = rint((phi_f - psi) / 2pi) in FP64 (half to
 * even), phi = (float)((double)psi + (double)K * 2pi).  ifg/is_complex/coh/mask
 * give psi and validity as in ww_integrate; phi_f NaN also counts as invalid.
 * unwrapped: DEVICE float32 [m][n] (NaN where invalid); cycles: DEVICE int32
 * [m][n] (0 where invalid).  Asynchronous. */
ww_status ww_transfer_cycles(const float* unwrapped_filtered, const void* ifg, int32_t is_complex, const float* coh,
                             const uint8_t* mask, int64_t m, int64_t n, float* unwrapped, int32_t* cycles,
                             ww_stream stream);

/* ---- Batched form: many uneven interferograms in one solve ----
 * Each item is one unwrap request (device pointers; outputs unwrapped/cycles are
 * m x n).  All items are solved together: their node grids are independent
 * (no arcs between items) and they share one free ground node, which leaves
 * each item's optimum unchanged because every item's supplies sum to zero.
 * One launch per grid step (residues, costs, integration) covers every item,
 * and one persistent search launch per pass covers the tiles of all unfinished
 * items; with params->graph_loop the whole pass loop is a single CUDA graph
 * launch whose loop condition is set on the device.
 * On return total_cost and status are filled in for every item. */
typedef struct ww_batch_item {
  const void* ifg;        /* float32 phase or interleaved complex64 [m][n] */
  int32_t is_complex;
  const float* coh;       /* [m][n] */
  const uint8_t* mask;    /* [m][n] or NULL */
  int64_t m, n;
  double nlooks;
  float* unwrapped;       /* out [m][n] */
  int32_t* cycles;        /* out [m][n] */
  int64_t total_cost;     /* out (host field) */
  int32_t status;         /* out (host field) */
} ww_batch_item;

typedef struct ww_batch ww_batch;  /* library-owned device scratch for batches */
/* Capacity: up to max_items items with at most max_pixels pixels in total and
 * max_item_pixels pixels in the largest item. */
ww_status ww_batch_create(int64_t max_items, int64_t max_pixels, int64_t max_item_pixels, ww_batch** out);
void ww_batch_free(ww_batch* b);
int64_t ww_batch_bytes(int64_t max_items, int64_t max_pixels, int64_t max_item_pixels);
/* Synchronises the stream; returns the first non-OK item status, else WW_OK. */
ww_status ww_unwrap_batch(ww_batch_item* items, int64_t count, const ww_params* params, ww_batch* b,
                          ww_stream stream);
/* Solver statistics of the last ww_unwrap_batch (all items together).  With
 * params->graph_loop (and WW_TRACE unset) the whole batch is one graph launch:
 * the three timing fields are then 0 and residues is 0 (only the device
 * counters are read back after the launch). */
ww_status ww_batch_stats(const ww_batch* b, ww_solve_stats* out);

/* Autotuner of the search schedule (no counterpart in the paper, whose CPU
 * solver has fixed settings).  Unwraps `items` (a sample of the workload to
 * tune for) with the starting parameters, then walks the knobs one at a time
 * (full_passes, band_start_ppm, band_min, band_mult, band_growth,
 * ground_sink_below, zero_stop_below, zero_band_hops, zero_band_hops_min,
 * search CTAs per SM, graph loop), keeping a value when it lowers the device time of the whole batched
 * unwrap (CUDA events, best of `repeats` runs).  Every trial must reproduce the
 * first trial's total cost for every item (the optimum is unique in cost even
 * where flows tie); otherwise WW_ERR_INTERNAL.  *best receives the chosen
 * parameters (all other fields copied from *start, or the defaults).  The
 * items' outputs are overwritten.  Synchronises the stream. */
typedef struct ww_tune_report {
  int32_t trials;
  float default_ms;   /* device time with *start */
  float best_ms;      /* device time with *best */
  int32_t reserved[5];
} ww_tune_report;
ww_status ww_autotune_batch(ww_batch_item* items, int64_t count, const ww_params* start, ww_batch* b,
                            int32_t repeats, ww_params* best, ww_tune_report* report, ww_stream stream);

/* ---- Served form: continuous batching ----
 * A server owns a worker thread, a CUDA stream and one running multi-problem
 * solve.  Submitted requests wait in FIFO order; between solver passes the
 * worker admits as many as the device-memory budget and max_active allow
 * (residues and costs computed on admission, state kept resident), retires the
 * requests whose imbalance reached zero (integration into the caller's output
 * buffers, total cost, status) and runs the next pass over all requests in
 * flight, so new requests join while others are on the GPU.  A request's device
 * buffers (ww_batch_item fields) must hold their inputs when it is submitted
 * and stay valid until it completes.  Requests larger than max_request_pixels
 * or than the budget are rejected at submit (WW_ERR_INVALID_ARG).
 * Every device allocation of the server (request state, batch tables, solver
 * state) is counted against hbm_budget_bytes: the server sizes its pools to
 * the largest that fits, and ww_server_create returns WW_ERR_INVALID_ARG when
 * the budget cannot hold one request of max_request_pixels. */
typedef struct ww_server_config {
  int64_t hbm_budget_bytes;   /* all device memory the server may allocate */
  int64_t max_request_pixels; /* largest request accepted */
  int32_t max_active;         /* requests in flight at once */
  int32_t reserved[7];
} ww_server_config;
typedef struct ww_server ww_server;
typedef struct ww_server_stats {
  int64_t submitted, admitted, completed, rejected, passes, peak_active;
  int64_t peak_resident_bytes;  /* device bytes the server allocated (<= hbm_budget_bytes) */
  double busy_ms;
} ww_server_stats;
ww_status ww_server_create(const ww_server_config* cfg, const ww_params* params, ww_server** out);
/* Queue a request; *ticket identifies it. */
ww_status ww_server_submit(ww_server* s, const ww_batch_item* req, int64_t* ticket);
/* *done = 1 once finished; then result->total_cost / status and *latency_ms
 * (submit to completion) are filled in (result and latency_ms may be NULL). */
ww_status ww_server_poll(ww_server* s, int64_t ticket, int32_t* done, ww_batch_item* result, double* latency_ms);
/* Block until the ticket finishes or timeout_ms passes (WW_ERR_TIMEOUT). */
ww_status ww_server_wait(ww_server* s, int64_t ticket, double timeout_ms, ww_batch_item* result,
                         double* latency_ms);
/* Forget a finished ticket. */
ww_status ww_server_release(ww_server* s, int64_t ticket);
ww_status ww_server_get_stats(ww_server* s, ww_server_stats* out);
/* Finishes the requests already submitted, then stops. */
void ww_server_destroy(ww_server* s);

/* ---- Harness: optimality certificate on the GPU ----
 * Counts violations into counts (device int64[4]): [0] |dk|>1 or flow on a
 * non-existent edge, [1] nodes (G included) whose out-in flow differs from the
 * supply, [2] residual arcs with negative reduced cost, [3] total cost. */
ww_status ww_certificate(const int8_t* residues, const int32_t* ground, const int16_t* costs,
                         const int8_t* flows, const int64_t* potentials, int64_t m, int64_t n,
                         int64_t* counts, ww_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* WW_H */
