// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ww.h"

namespace ww {

// ---- fp32 constants of the specified formulas (bit patterns in comments) ----
constexpr float kPiF = 3.14159274101257324f;        // 0x40490FDB
constexpr float kTwoPiF = 6.28318548202514648f;     // 0x40C90FDB
constexpr float kAlphaScale = 40.7436637878417969f; // fp32(256/(2pi)), 0x4222F983
constexpr double kTwoPiD = 6.283185307179586;       // 0x1.921fb54442d18p+2
constexpr int kNGamma = 128;
constexpr int kNAlpha = 256;
constexpr float kQScale = 4194304.0f;               // 2^22 fixed point for the slope sum

// ---- search label packing: d (32 bits) | hops (29 bits) | dir (3 bits) ----
constexpr uint64_t kInf = ~0ull;
constexpr int kDirRoot = 0, kDirUp = 1, kDirDown = 2, kDirLeft = 3, kDirRight = 4;
constexpr uint32_t kNoArc = 0xFFFFFFFFu;  // reduced cost of a missing residual arc

#if defined(__CUDACC__)
__host__ __device__ inline uint32_t label_dist(uint64_t k) { return (uint32_t)(k >> 32); }
__host__ __device__ inline int label_dir(uint64_t k) { return (int)(k & 7); }

// Fixed-point CORDIC atan2, the phase of a complex sample: the two fp32 parts
// scaled exactly to integers with the larger below 2^30, a quadrant step, then
// 30 vectoring iterations with angle unit 2^-29 rad; table entries are
// round(atan(2^-i) 2^29).  Integer-only, so every build gives the same bits.
static __constant__ int32_t kAtanQ[30] = {
    421657428, 248918915, 131521918, 66762579, 33510843, 16771758, 8387925, 4194219,
    2097141,   1048575,   524288,    262144,   131072,   65536,    32768,    16384,
    8192,      4096,      2048,      1024,     512,      256,      128,      64,
    32,        16,        8,         4,        2,        1};
constexpr int64_t kHalfPiQ = 843314857;  // round(pi/2 * 2^29)

// a b + c mod 2^32 (an integer multiply-add; no overflow rules of C++ apply).
__device__ __forceinline__ int32_t mad32(int32_t a, int32_t b, int32_t c) {
  int32_t d;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// |v| = M 2^E for a finite fp32 value (M < 2^24), with its sign bit.
__device__ __forceinline__ void f32_split(float v, int32_t* M, int* E, int* neg) {
  uint32_t b = __float_as_uint(v);
  *neg = (int)(b >> 31);
  int be = (int)((b >> 23) & 0xFF);
  uint32_t fr = b & 0x7FFFFFu;
  *M = (int32_t)(be == 0 ? fr : (fr | 0x800000u));
  *E = be == 0 ? -149 : be - 150;
}

// M 2^(E + 30 - top) truncated toward zero, negated when neg.  top is the
// larger component's E + bit length, so the shift never exceeds 29 and the
// larger component lands in [2^29, 2^30): every result fits 32 bits.
__device__ __forceinline__ int32_t fixed_scale(int32_t M, int E, int top, int neg) {
  int sh = E + 30 - top;
  int32_t r = sh >= 0 ? (sh >= 31 ? 0 : (M << sh)) : (-sh >= 24 ? 0 : (M >> (-sh)));
  return neg ? -r : r;
}

__device__ __forceinline__ float cordic_phase(float re, float im) {
  int32_t Mx, My;
  int Ex, Ey, nx, ny;
  f32_split(re, &Mx, &Ex, &nx);
  f32_split(im, &My, &Ey, &ny);
  if ((Mx | My) == 0) return 0.0f;
  int tx = Mx ? Ex + (32 - __clz(Mx)) : -100000;
  int ty = My ? Ey + (32 - __clz(My)) : -100000;
  int top = max(tx, ty);
  int32_t X = fixed_scale(Mx, Ex, top, nx);
  int32_t Y = fixed_scale(My, Ey, top, ny);
  int32_t Z = 0;
  if (X < 0) {
    int32_t t = X;
    if (Y >= 0) {
      X = Y;
      Y = -t;
      Z = (int32_t)kHalfPiQ;
    } else {
      X = -Y;
      Y = t;
      Z = -(int32_t)kHalfPiQ;
    }
  }
  // Vectoring iterations in 32-bit registers.  With |X|, |Y| < 2^30 and X >= 0
  // here, X only grows, to at most the CORDIC gain (1.647) times |(X, Y)| <
  // 2^32 (unsigned); |Y| stays below max(|Y|, X >> i) < 2^31; |Z| <= pi 2^29.
  // Each step, branch-free with g = sign(Y) as +-1 (Y = 0 counts as +):
  // X += g (Y >> i) (= |Y >> i| as the arithmetic shift rounds), Y -= g (X >> i),
  // Z += g atan(2^-i).  The products by g are integer multiply-adds (wrapping
  // mod 2^32, the same bits as negating) and X >> i a multiply-high by
  // 2^(32-i), which keeps half of each step off the integer ALU.
  uint32_t x = (uint32_t)X;
  int32_t y = Y, z = Z;
#pragma unroll
  for (int i = 0; i < 30; ++i) {
    const int32_t s = y >> 31;
    const int32_t g = s | 1, ng = ~s | 1;
    const uint32_t xs = i == 0 ? x : __umulhi(x, 1u << (32 - i));
    x = (uint32_t)mad32(y >> i, g, (int32_t)x);
    y = mad32((int32_t)xs, ng, y);
    z = mad32(kAtanQ[i], g, z);
  }
  float psi = __fmul_rn(__int2float_rn(z), 1.0f / 536870912.0f);
  return fminf(fmaxf(psi, -kPiF), kPiF);
}

// Fixed-point CORDIC rotation: (cos t, sin t) scaled to length 2^30 for the
// angle t = Z 2^-29 rad, |Z| <= round(pi 2^29).  The start vector is
// (K^-1 2^30, 0) with K^-1 = prod over the 30 steps of (1 + 2^-2i)^(-1/2), so the
// rotation gain brings it to length 2^30; angles beyond +-pi/2 are first turned
// by a quarter turn; step i turns by -+atan(2^-i) toward Z = 0.  |X|, |Y| stay
// below 2^30 (the length only grows toward 2^30) and |Z| below 2^31.
constexpr int32_t kInvGainQ30 = 652032874;  // round(2^30 prod (1 + 2^-2i)^(-1/2)), i < 30

__device__ __forceinline__ void cordic_cos_sin(int32_t z, int32_t* c, int32_t* s) {
  int32_t x = kInvGainQ30, y = 0;
  if (z > (int32_t)kHalfPiQ) {
    x = 0;
    y = kInvGainQ30;
    z -= (int32_t)kHalfPiQ;
  } else if (z < -(int32_t)kHalfPiQ) {
    x = 0;
    y = -kInvGainQ30;
    z += (int32_t)kHalfPiQ;
  }
  // each step with h = +1 for Z >= 0, -1 otherwise: X -= h (Y >> i),
  // Y += h (X >> i), Z -= h atan(2^-i), the products as multiply-adds
#pragma unroll
  for (int i = 0; i < 30; ++i) {
    const int32_t xs = x >> i, ys = y >> i;
    const int32_t s = z >> 31;
    const int32_t h = s | 1, nh = ~s | 1;
    x = mad32(ys, nh, x);
    y = mad32(xs, h, y);
    z = mad32(kAtanQ[i], nh, z);
  }
  *c = x;
  *s = y;
}

// Interpolated cost (cost_lookup = 1): bilinear in the table of 100 ln(P0/P+)
// at the bin centres, fp32 with every operation rounded once, then floor and
// saturation to [0, 32767].
__device__ __forceinline__ int16_t bilinear_cost(const float* __restrict__ ratio, float a, float g) {
  const float x = __fsub_rn(__fmul_rn(__fadd_rn(a, kPiF), kAlphaScale), 0.5f);
  const float y = __fsub_rn(__fmul_rn(g, 128.0f), 0.5f);
  const int j0 = min(254, max(0, (int)floorf(x)));
  const int k0 = min(126, max(0, (int)floorf(y)));
  const float fx = fminf(1.0f, fmaxf(0.0f, __fsub_rn(x, (float)j0)));
  const float fy = fminf(1.0f, fmaxf(0.0f, __fsub_rn(y, (float)k0)));
  const float* r0 = ratio + k0 * kNAlpha + j0;
  const float a00 = __ldg(r0), a01 = __ldg(r0 + 1), a10 = __ldg(r0 + kNAlpha), a11 = __ldg(r0 + kNAlpha + 1);
  const float v0 = __fadd_rn(a00, __fmul_rn(fx, __fsub_rn(a01, a00)));
  const float v1 = __fadd_rn(a10, __fmul_rn(fx, __fsub_rn(a11, a10)));
  const float v = __fadd_rn(v0, __fmul_rn(fy, __fsub_rn(v1, v0)));
  if (!(v > 0.0f)) return 0;
  if (v >= 32767.0f) return 32767;
  return (int16_t)floorf(v);
}

// Wrap count of a phase difference (fp32): +1 above pi, -1 at or below -pi.
__device__ __forceinline__ int wrap_count(float dpsi) {
  return (dpsi > kPiF ? 1 : 0) - (dpsi <= -kPiF ? 1 : 0);
}

// Load one pixel's prepared phase and validity (invalid -> psi 0).
struct Pix {
  float psi;
  float coh;
  bool valid;
};

__device__ __forceinline__ Pix load_pixel(const void* ifg, int is_complex, const float* coh,
                                          const uint8_t* mask, int64_t k) {
  Pix p;
  bool ok = mask ? (__ldg(mask + k) != 0) : true;
  float c = coh ? __ldg(coh + k) : 1.0f;
  ok = ok && isfinite(c);
  float psi;
  if (is_complex) {
    float2 z = __ldg(reinterpret_cast<const float2*>(ifg) + k);
    ok = ok && isfinite(z.x) && isfinite(z.y);
    psi = ok ? cordic_phase(z.x, z.y) : 0.0f;
  } else {
    float v = __ldg(reinterpret_cast<const float*>(ifg) + k);
    ok = ok && isfinite(v);
    psi = ok ? v : 0.0f;
  }
  p.psi = ok ? psi : 0.0f;
  p.coh = ok ? c : 0.0f;
  p.valid = ok;
  return p;
}

// LUT indices: fp32, every operation rounded separately.
__device__ __forceinline__ int alpha_index(float a) {
  float t = __fmul_rn(__fadd_rn(a, kPiF), kAlphaScale);
  int k = (int)floorf(t);
  return min(255, max(0, k));
}
__device__ __forceinline__ int gamma_index(float g) {
  int k = (int)floorf(__fmul_rn(g, 128.0f));
  return min(127, max(0, k));
}
#endif  // __CUDACC__

}  // namespace ww

// ---- host-side objects ----
struct ww_lut {
  double nlooks;
  void* shared;  // LutData* (see ww_api.cu)
};

namespace ww {
// Device state of the MCF solver for up to n_cap nodes, t_cap 32x32 tiles and
// p_cap problems (ww_mcf.cu).
struct SolverWs {
  int64_t n_cap, t_cap, p_cap;
  int32_t* excess;     // [n_cap] imbalance per node
  uint64_t* labels;    // [n_cap] search labels (distance | hops | direction)
  uint64_t* best;      // [n_cap] per tree root: nearest candidate (distance, id)
  int32_t* cand;       // [2 n_cap] current / next list of imbalanced nodes
  int32_t* cand_root;  // [n_cap]
  int64_t* pot;        // [n_cap + 1] potentials when the caller's array is not used; last = ground
  int32_t* inq;        // [t_cap] 1 while a tile is queued
  int32_t* slots;      // [t_cap + ring slack] worklist ring (tile + 1, 0 = empty)
  int32_t* capped;     // [t_cap] tile dropped a candidate at the distance cap
  int32_t* touched;    // [t_cap] 1 once the search visited the tile in this pass
  int32_t* tlist;      // [t_cap] tiles the search visited in this pass
  // reduced arc costs of tiles 0 .. rc_entries-1 in the current pass ([rc_entries][4][32][32]),
  // and the pass + 1 whose costs an entry holds (0: none); tiles beyond are not cached
  int64_t rc_entries;
  uint32_t* rc_cache;
  int32_t* rc_pass;
  uint16_t* exits;     // [n_cap] per node reached in the pass: tile-local index where its parent chain leaves the tile
  int32_t* segs;       // [n_cap] first nodes of the tile segments of a pass's augmenting paths
  int32_t* tile_prob;  // [t_cap] tile -> problem
  int32_t* border;     // border tiles of every problem
  void* probs;         // ProbDev [p_cap]
  void* host_probs;    // pinned ProbDev [p_cap]
  int32_t* prob_left;  // [p_cap] imbalanced nodes per problem
  long long* g_net;    // [p_cap] net units emitted by the ground node per problem
  long long* tc;       // [p_cap] total cost per problem
  int32_t* order;      // [p_cap] active slots by node offset
  int32_t* slot_list;  // [p_cap] scratch list of slots for per-problem launches
  int32_t* status_all; // [p_cap] statuses of a finalize call
  void* ctr;           // McfCtr
  void* q;             // SearchQ
  void* host_ctr;      // pinned McfCtr mirror
  void* events[2];     // search timing
  // pinned staging of the host-built lists (so uploads can sit in a CUDA graph):
  // order [p_cap] | border [nb_cap] | joiners [p_cap] | finalize list [p_cap] | statuses [p_cap]
  int32_t* h_lists;
  int64_t nb_cap;
};

// One problem handed to the solver (all pointers on the device).
struct ProbHost {
  int64_t m, n;
  const int8_t* res;
  const int32_t* ground;
  const int16_t* costs;
  int8_t* flows;
  int64_t* pot_out;
  int64_t* total_cost;
  int32_t* status;
  // start from the flows already in `flows` and the potentials already in the
  // solver's potential array (single problem with the caller's potentials only)
  bool resume = false;
};
}  // namespace ww

struct ww_workspace {
  int device;
  int64_t max_rows, max_cols;
  ww::SolverWs sv;
  // path scratch for ww_unwrap
  int8_t* residues;
  int32_t* ground;
  int16_t* costs;
  int8_t* flows;
  int64_t* potentials;
  int64_t* total_cost;
  int32_t* dev_status;
  // steep selection scratch
  uint32_t* hist;       // [65536]
  uint64_t* steep_ctr;  // [8]
  uint32_t* blocksum;   // per-block tie counts
  int64_t blocksum_len;
  uint32_t* steep_list;  // keys of the steep candidates (while within capacity)
  int64_t steep_list_cap;
  float* psi;            // wrapped phase of a complex input, computed once per unwrap
  // statistics of the last solve
  ww_solve_stats stats;
};

#define WW_CUDA_TRY(expr)                          \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return WW_ERR_CUDA;     \
  } while (0)

namespace ww {
// ww_lut.cpp
int lut_build_host(double nlooks, int16_t* table, double* cost100, float* ratio100);
// ww_api.cu
const int16_t* lut_device_table(const ww_lut* lut, cudaStream_t stream, ww_status* st);
// device copy of the fp32 table of 100 ln(P0/P+) (interpolated lookup), or null
// with *st = WW_ERR_INVALID_ARG when the table object carries none
const float* lut_device_ratio(const ww_lut* lut, ww_status* st);
const int16_t* lut_host_table(const ww_lut* lut);
// page-locked copy of the host table, or null if it could not be made
const int16_t* lut_pinned_table(const ww_lut* lut);
// ww_grid.cu
ww_status launch_residues(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                          int64_t m, int64_t n, int8_t* res, int32_t* ground, cudaStream_t s);
ww_status launch_costs(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                       int64_t m, int64_t n, const int16_t* dtable, const float* dratio, const ww_params* p,
                       ww_workspace* ws, int16_t* costs, cudaStream_t s, int8_t* res = nullptr,
                       int32_t* ground = nullptr);
// (res, ground given: the residues of Eq. 1 and the ground charge are written by
// the same tiles; *ground must be zero before the call)
ww_status launch_integrate(const void* ifg, int is_complex, const float* coh, const uint8_t* mask,
                           const int8_t* flows, int64_t m, int64_t n, float* unw, int32_t* cyc,
                           cudaStream_t s);
// psi[k] = CORDIC phase of a complex64 image, NaN where a sample is not finite
// and (when given) where the mask is 0 or the coherence is not finite
ww_status launch_phase(const void* ifg, const float* coh, const uint8_t* mask, int64_t m, int64_t n, float* psi,
                       cudaStream_t s);
// Connected-component labels over reliable edges (ww_cc.cu).
ww_status launch_components(const int16_t* costs, const int8_t* flows, const float* unwrapped, int64_t m, int64_t n,
                            int32_t threshold, int32_t* labels, cudaStream_t s);
// candidate-list entries needed for an image of `pixels` pixels at cap_ppm (cap + 2)
int64_t steep_list_capacity(int64_t pixels, int32_t cap_ppm);
// Batched launches of the grid steps (ww_grid.cu): one launch per step covers
// every item; blk[] holds each item's first block per launch kind.
enum { kBlkRes = 0, kBlkCost = 1, kBlkSteep = 2, kBlkRow = 3, kBlkSel = 4, kBlkPhase = 5, kBlkKinds = 6 };
struct GridItem {
  const void* ifg;
  const float* coh;
  const uint8_t* mask;
  int64_t m, n;
  int32_t is_complex, pad;
  int64_t blk[kBlkKinds];
  int8_t* res;
  int32_t* ground;
  int16_t* costs;
  const int16_t* table;
  const float* ratio;  // 100 ln(P0/P+) table of the interpolated lookup (null otherwise)
  void* steep;  // per-item steep-selection counters (set by launch_pre_batch)
  uint32_t* cand_list;  // steep candidate keys (set by launch_pre_batch; null: no list)
  int64_t cand_cap;
  const void* phase_src;  // complex64 image whose phase launch_pre_batch writes into ifg (a float
                          // buffer, is_complex 0), or null
  const int8_t* flows;
  float* unw;
  int32_t* cyc;
};
struct GridBatch {
  GridItem* d_items = nullptr;
  GridItem* h_items = nullptr;  // pinned; filled by the caller (all but blk and steep)
  void* d_steep = nullptr;      // per-item steep counters
  uint32_t* hist = nullptr;     // per-item selection histograms (2048 bins)
  uint32_t* blocksum = nullptr; // per-chunk tie counts of the selection
  int64_t blocksum_len = 0;
  uint32_t* list_pool = nullptr; // steep candidate lists of all items
  int64_t list_pool_cap = 0;
  int cap = 0;
};
int64_t grid_batch_bytes(int cap, int64_t max_pixels);
ww_status grid_batch_alloc(GridBatch* gb, int cap, int64_t max_pixels);
void grid_batch_free(GridBatch* gb);
// residues + costs (with the steep rule, exact selection for the items over
// their cap) of items [0, count): a fixed number of launches, no host sync.
// Items with phase_src get their phase computed once into ifg first.
ww_status launch_pre_batch(GridBatch* gb, int count, const ww_params* p, cudaStream_t s);
// integration of items [0, count) (fields ifg, coh, mask, m, n, is_complex,
// flows, unw, cyc of h_items); uploads the item table
ww_status launch_integrate_batch(GridBatch* gb, int count, cudaStream_t s);
// The item table is copied from pinned host memory asynchronously: h_items must
// not be rewritten before the stream has passed the launch that used it.
// ww_mcf.cu
struct Batch;
struct McfCtr;
// A solve over a changing set of problems: problems join (add + commit) and
// leave (finalize + remove) between passes; passes alternate forward/reverse.
// All problems share the free ground node (potential at pot[g_index]).
class Session {
 public:
  Session(SolverWs* sv, int64_t* pot, int64_t g_index, const ww_params* prm, cudaStream_t s,
          bool keep_ground_pot = false);
  int next_slot() const;                                            // slot the next add() takes, -1 if full
  int add(const ProbHost& ph, int64_t node_off, int64_t tile_off);  // -> slot, or -1 if full
  void remove(int slot);
  ww_status commit();                                               // upload layout, initialise joiners
  ww_status pass(ww_solve_stats* st);                               // one pass, then a host sync
  ww_status run_graph(ww_solve_stats* st);  // all remaining passes in one graph launch (device-driven loop)
  ww_status left(std::vector<int32_t>* out);                        // imbalanced nodes per slot
  ww_status finalize(const std::vector<int>& slots, std::vector<int32_t>* statuses);
  // finalize without the host sync: statuses land in finalized_status() once the stream has passed
  ww_status finalize_enqueue(const std::vector<int>& slots);
  const int32_t* finalized_status() const;
  // the remaining passes as one conditional while node of graph g (after dep, if any)
  ww_status add_loop_node(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraphNode_t* out);
  void set_stream(cudaStream_t s) { stream = s; }
  cudaStream_t get_stream() const { return stream; }
  // the host does not know the number of imbalanced nodes (whole-graph capture)
  void set_ncand_unknown(bool v) { ncand_unknown = v; }
  void fill_stats(ww_solve_stats* st) const;  // counters from the host mirror of the device state
  int64_t ctr_bytes() const;                   // size of the device counter block (host mirror)
  const McfCtr& ctr() const;
  int32_t status() const;
  int32_t ncand() const;
  bool go_on() const;
  int64_t tiles_of(int slot) const;
  ww_status err = WW_OK;

 private:
  template <bool FWD>
  ww_status enqueue_pass();
  Batch batch() const;
  SolverWs* sv;
  int64_t* pot;
  int64_t g_index;
  cudaStream_t stream;
  int sm_count = 148, search_grid = 592;
  std::vector<char> used;
  std::vector<int> order, pending;
  int64_t n_total = 0, t_high = 0, max_nodes = 1, n_border = 0, max_garcs = 1;
  int parity = 0;
  bool capturing = false;  // enqueue_pass is being captured into a graph body
  bool staged_zero = false;  // the zero band's hop radius grows in stages
  bool ncand_unknown = false;
};

// argument check of a ww_params (ww_api.cu)
bool params_valid(const ww_params* p);
// WW_TRACE=1 in the environment: per-pass and per-phase timings on stderr
bool trace_enabled();
ww_status solve_problems(const ProbHost* probs, int nprob, SolverWs* sv, const ww_params* prm, int64_t* pot_global,
                         ww_solve_stats* stats, cudaStream_t s);
ww_status launch_certificate(const int8_t* res, const int32_t* ground, const int16_t* costs,
                             const int8_t* flows, const int64_t* pot, int64_t m, int64_t n,
                             int64_t* counts, cudaStream_t s);
int64_t solver_bytes(int64_t n_nodes, int64_t n_tiles, int64_t n_probs);
ww_status solver_alloc(SolverWs* sv, int64_t n_nodes, int64_t n_tiles, int64_t n_probs);
void solver_free(SolverWs* sv);
inline int64_t tiles_for(int64_t m, int64_t n) { return ((m - 1 + 31) / 32) * ((n - 1 + 31) / 32); }
}  // namespace ww
