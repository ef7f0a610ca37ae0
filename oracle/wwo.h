/* CPU oracle for the Whirlwind MCF unwrapper hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C++ that restates the
 * paper's definitions so the CUDA library can be checked against it.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code with the CUDA library.
 *
 * Conventions (all arrays row-major, m rows x n cols of pixels):
 *   h(i,j): pixel edge (i,j)->(i,j+1), stored at [i*n+j] of an m x n plane.
 *   v(i,j): pixel edge (i,j)->(i+1,j), stored at [i*n+j] of an m x n plane.
 *   Dual node p=(i,j), 0<=i<m-1, 0<=j<n-1, index i*(n-1)+j; the ground node G
 *   (collapsed outer ring, Sec. II-A) has index (m-1)*(n-1).
 *   h(i,j) separates node (i-1,j) [above] from (i,j) [below]; v(i,j) separates
 *   node (i,j-1) [left] from (i,j) [right]; nodes outside the grid are G.
 *   Cost planes [4][m][n]: 0 = above->below across h (gives dk_h=+1),
 *   1 = below->above across h (dk_h=-1), 2 = right->left across v (dk_v=+1),
 *   3 = left->right across v (dk_v=-1).
 *   Flow planes [2][m][n] int8: dk_h, dk_v in {-1,0,1}.
 */
#ifndef WWO_H
#define WWO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- inputs ---- */
/* psi = own CORDIC atan2(im, re) for interleaved complex64 (count pixels). */
void wwo_phase_from_complex(const float* ifg, int64_t count, float* psi);
/* Validity and masked replacement: valid = mask!=0 && finite inputs; masked
 * pixels get psi = 0, coh = 0.  ifg (interleaved) or phase must be non-null. */
void wwo_prepare(const float* phase, const float* ifg, const float* coh, const uint8_t* mask,
                 int64_t m, int64_t n, float* psi, float* coh_out, uint8_t* valid);

/* ---- Eq. (1) residues ---- */
void wwo_residues(const float* psi, int64_t m, int64_t n, int8_t* res, int32_t* ground);

/* ---- Sec. II-B arc costs ---- */
/* alpha-hat of every valid edge (0 where invalid): planes [2][m][n] (h, v). */
void wwo_alpha_hat(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t half_width,
                   float* alpha);
/* Full cost planes from a 128 (gamma) x 256 (alpha) int16 table. Returns the
 * number of steep edges zeroed. */
int64_t wwo_costs(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                  const int16_t* table, int32_t half_width, float steep_rad, int32_t steep_cap_ppm,
                  int16_t* costs);
/* Cost-model variants: slope_mode 0 = fixed-point mean of wrapped gradients,
 * 1 = argument of the sum of unit phasors (CORDIC); lookup 0 = nearest bin of
 * the int16 table, 1 = bilinear interpolation of the float table ratio
 * (100 ln(P0/P+) at the bin centres, 128 x 256) then floor, saturated. */
int64_t wwo_costs2(const float* psi, const float* coh, const uint8_t* valid, int64_t m, int64_t n,
                   const int16_t* table, const float* ratio, int32_t half_width, int32_t slope_mode,
                   int32_t lookup, float steep_rad, int32_t steep_cap_ppm, int16_t* costs);
void wwo_alpha_hat2(const float* psi, const uint8_t* valid, int64_t m, int64_t n, int32_t half_width,
                    int32_t mode, float* alpha);

/* ---- preprocessing: multilook + Eq. (3) sample coherence ----
 * slc1, slc2: interleaved complex64 [M][N]; outputs [M/ly][N/lx]: ifg
 * (interleaved complex64, sum z1 conj(z2)) and coh (float32).  fp32, fixed order. */
void wwo_multilook(const float* slc1, const float* slc2, int64_t M, int64_t N, int32_t ly, int32_t lx,
                   float* ifg, float* coh);

/* ---- integration ---- */
void wwo_integrate(const float* psi, const uint8_t* valid, const int8_t* flows, int64_t m, int64_t n,
                   float* unwrapped, int32_t* cycles);

/* ---- Eq. (2) MCF ---- */
/* status: 0 ok, -4 infeasible.  potentials has (m-1)(n-1)+1 entries. */
int wwo_solve_mcf(const int8_t* res, int32_t ground, const int16_t* costs, int64_t m, int64_t n,
                  int8_t* flows, int64_t* potentials, int64_t* total_cost);
/* 0 ok; 1 capacity; 2 conservation; 3 negative reduced cost on a residual arc. */
int wwo_check_certificate(const int8_t* res, int32_t ground, const int16_t* costs, int64_t m,
                          int64_t n, const int8_t* flows, const int64_t* potentials,
                          int64_t* total_cost, int64_t* bad_index);
/* Cost of a flow (sum of c_a x_a); -1 if some |dk|>1. */
int64_t wwo_flow_cost(const int16_t* costs, int64_t m, int64_t n, const int8_t* flows);
/* Exhaustive minimum over integer cycle maps K (K(0,0)=0, |dk|<=1), m*n <= 30. */
int64_t wwo_brute_force(const float* psi, const int16_t* costs, int64_t m, int64_t n);
/* 1 if the supplies can be routed within unit capacities (max-flow), else 0. */
int wwo_feasible(const int8_t* res, int32_t ground, int64_t m, int64_t n);

/* ---- FP64 cost tables (Eqs. 4-7) ---- */
double wwo_lee_pdf(double eta, double gamma, double L);
double wwo_touzi_pdf(double gh, double gamma, double L);
/* Coherence-marginalised phase pdf (Eq. 5) on eta_k = -pi + k*pi/nh, k=0..2nh. */
int wwo_marginal_pdf(double L, double gh, int32_t nh, int32_t lambda_panels, double* f);
/* sigma_alpha from a tabulated single-pixel pdf on the same grid. */
double wwo_sigma_from_pdf(const double* f, int32_t nh);
/* P0, P+ for one (alpha-hat, gamma-hat) from a tabulated pdf. */
void wwo_probabilities(const double* f, int32_t nh, double alpha_hat, double* p0, double* pplus,
                       double* pminus, double* sigma);
/* The whole 128 x 256 table: 100*c in FP64 (cost100), floor'd int16, and
 * (ratio100, may be NULL) 100 ln(P0/P+) in fp32 for interpolated lookup. */
int wwo_lut_build(double L, int32_t nh, int32_t lambda_panels, double* cost100, int16_t* table, float* ratio100);

#ifdef __cplusplus
}
#endif
#endif
