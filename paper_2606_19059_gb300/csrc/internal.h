// internal.h -- plan layout and kernel launchers of the GB300 spectral Ewald
// library.  Private to the library; the public ABI is include/ewald_gb300.h.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>
#include <cmath>

#include <vector>

#include "../../include/ewald_gb300.h"

struct CUtensorMap_st;  // the driver API's TMA descriptor (cuda.h), used by the grid kernels

namespace ewg {

// 32-byte FP64 quadruple (CUDA 13 deprecates double4)
struct __align__(32) dvec4 {
    double x, y, z, w;
};

// A coordinate wrapped into [0, L) the way binning places points: positions
// already inside are left as they are (inv_L = 1.0 / L).
__host__ __device__ inline double wrap_coord(double v, double L, double inv_L)
{
    if (v < 0.0 || v >= L) {
        v -= L * floor(v * inv_L);
        if (v >= L)
            v -= L;
    }
    if (v < 0.0)
        v = 0.0;
    return v;
}

constexpr int kSub = 2;             // sub-cells per near cell per side (target ordering)
constexpr int kSub3 = kSub * kSub * kSub;
constexpr int kMaxP = 16;           // largest window support the kernels implement
constexpr int kMaxDeg = 20;         // largest window polynomial degree
constexpr int kNumEvents = 10;
constexpr int kP2PChunk = 32;       // targets per P2P work item (one warp)
constexpr int kGridDsMinP = 8;      // smallest support of the double-single grid kernels

// P2P work items are cut from groups of cells: two x-neighbours when the
// cutoff reaches one cell (K = 1; a warp's 32 targets may straddle them, so
// warps stay full), single cells when it reaches two (K = 2).  Groups run
// along x in each row (y, z); with odd n_c a row ends on a one-cell group.
__host__ __device__ inline int p2p_group_cells(int K) { return K == 1 ? 2 : 1; }
__host__ __device__ inline int p2p_groups_per_row(int nc, int K)
{
    return (nc + p2p_group_cells(K) - 1) / p2p_group_cells(K);
}
__host__ __device__ inline int p2p_groups(int nc, int K) { return nc * nc * p2p_groups_per_row(nc, K); }
// first cell of group g and its number of cells
__host__ __device__ inline int p2p_group_cell(int g, int nc, int K, int &ncg)
{
    const int gpr = p2p_groups_per_row(nc, K), gc = p2p_group_cells(K);
    const int row = g / gpr, x0 = (g - row * gpr) * gc;
    ncg = nc - x0 < gc ? nc - x0 : gc;
    return row * nc + x0;
}

// The box of global block (or element) index g among many plans launched
// together: base[b] <= g < base[b + 1] (base holds nbox + 1 prefix offsets).
__device__ __forceinline__ int find_box(const int *base, int nbox, int g)
{
    int lo = 0, hi = nbox;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// double-single window weights: bins of one axis padded to a multiple of 4
inline int ds_window_stride(int P) { return (P + 3) & ~3; }

// Bank dealing for G2P from a staged grid block with row stride S (floats):
// lane b takes the (y, x) pairs of a P x P face with (S y + x) mod 32 = b, one
// per round.  g2p_rounds: the rounds that takes (the most pairs on one bank);
// g2p_stride: the S, from T + P - 1 (T = 8) rounded up to 4, with the fewest.
__host__ __device__ constexpr int g2p_rounds(int P, int S)
{
    int mx = 0;
    for (int b = 0; b < 32; ++b) {
        int cnt = 0;
        for (int yy = 0; yy < P; ++yy)
            if (((b - S * yy) & 31) < P)
                ++cnt;
        mx = cnt > mx ? cnt : mx;
    }
    return mx;
}
__host__ __device__ constexpr int g2p_stride(int P)
{
    const int s0 = (P + 7 + 3) & ~3;  // T + P - 1 rounded up to 4
    int best = s0, br = g2p_rounds(P, s0);
    for (int S = s0 + 4; S <= s0 + 8; S += 4) {
        const int r = g2p_rounds(P, S);
        if (r < br) {
            best = S;
            br = r;
        }
    }
    return best;
}

// Window polynomial for one precision: coef[l * (deg+1) + k] is the z^k
// coefficient of bin l, z = 2 delta - 1 (Sec. 2.2 / Sec. 4, Horner form).
struct WindowPoly {
    int P = 0, deg = 0;
    std::vector<double> coef;
};

struct Geometry {
    // near field
    int nc;              // cells per side
    int K;               // neighbour cell reach per side (1 when cell >= rc)
    double cell;         // cell width
    int ncells;          // nc^3
    int nkeys;           // ncells * kSub3
    // far field
    int M, P, T, nt;     // grid size, support, tile edge, tiles per side
    int ntiles;          // nt^3
    int KT;              // neighbour tile reach for P2G: ceil((P-1)/T)
    double h;
    int Mh;              // M/2 + 1
    int64_t nreal;       // M^3
    int64_t ncplx;       // M * M * Mh
};

}  // namespace ewg

struct ewald_plan_s {
    int device = -1;
    int64_t N = 0;
    ewald_dtype dtype = EWALD_F64;
    ewald_params prm{};
    ewg::Geometry g{};
    ewg::WindowPoly wpoly;
    bool near64 = true, fft64 = true;

    // binning state
    int32_t *keyn = nullptr, *slotn = nullptr, *keyt = nullptr, *slott = nullptr;
    int32_t *cntn = nullptr, *startn = nullptr;   // nkeys + 1
    int32_t *cntt = nullptr, *startt = nullptr;   // ntiles + 1
    int32_t *items = nullptr, *item_off = nullptr;  // P2P work items per cell (ncells + 1)
    int32_t *permn = nullptr, *permt = nullptr;   // sorted slot -> user index
    void *npos = nullptr, *nfrc = nullptr;        // near-sorted positions (cell-local) / forces
    void *nlo = nullptr;                          // (unused since the FP32 records)
    void *nrec = nullptr;                         // FP32: near-sorted 32-byte source records
    void *nflo = nullptr;                         // double-single: force low parts (float4)
    bool near_ds = false;                         // P2P in double-single arithmetic
    double ds_r1 = 0.0;                           // double-single P2P: pairs beyond this radius in FP32
    bool grid_ds = false;                         // P2G / G2P in double-single arithmetic
    void *wts = nullptr;                          // double-single window weights (tile order)
    void *tdat = nullptr, *tfrc = nullptr;        // tile-sorted window data / forces
    void *un = nullptr, *uf = nullptr;            // near / far results, user order
    void *grid = nullptr;                         // 3 M^3 real
    bool ext_grid = false;                        // grid and spec belong to a batch's grouped FFT
    void *grid_g2p = nullptr;                     // G2P input in the kernels' precision (may alias grid)
    bool own_grid_g2p = false;
    // double layer (Sec. 2.3), allocated by the first combined apply: the
    // tile-order symmetric densities (2 x N quadruples in the P2G input
    // precision), their two 3-component grids and half spectra
    void *dl_tf = nullptr, *dl_grid = nullptr, *dl_spec = nullptr;
    void *dl_near = nullptr;  // near-sorted positions, q, n (3 x N dvec4) and FP32 local hi, lo, q, n (4 x N float4)
    void *spec = nullptr;                         // 3 M^2 (M/2+1) complex
    void *tab = nullptr;                          // CNV 1-D table (M entries)
    void *wcoef_dev = nullptr;                    // window polynomial coefficients
    int *err = nullptr;                           // device error flag
    double *hx = nullptr, *hf = nullptr, *hu = nullptr;  // device staging for ewald_apply_host
    size_t scan_tmp_bytes = 0;

    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    // M in {64, 128, 256}: FP32 spectra, 2-D (y, x) transforms of the 3 M
    // planes around the fused z-FFT / CNV / z-IFFT kernels (k_fgc_z.cu; the
    // double layer's two density triples through the same 2-D plan); FP64
    // spectra, the Stokeslet alone, 1-D transforms along x of the 3 M^2 rows
    // around the double-single y and z kernels (k_fgc_z64.cu)
    cufftHandle fwd2 = 0, inv2 = 0;
    bool have_fwd2 = false, have_inv2 = false, fgc_fused = false;
    void *twz = nullptr;                          // w_M^j, j < M (FP32 complex; FP64 spectra:
                                                  // split h + l, then the CNV table split)
    void *fftwork = nullptr;                      // shared cuFFT work area (every plan)
    bool pooled = false;                          // workspaces from the stream-ordered pool
    cudaStream_t s2 = nullptr;                    // second stream: P2P alongside the far field
    cudaStream_t s3 = nullptr;                    // origin stream of the applies' graph captures
    struct GraphSlot {                            // a captured apply and the buffers it bakes in
        enum Mode { kUndecided, kGraph, kDirect };
        const void *a = nullptr, *b = nullptr, *c = nullptr;
        cudaGraphExec_t exec = nullptr;
        int calls = 0;                            // calls with these buffers (counted up to 3)
        Mode mode = kUndecided;                   // replay or direct launches, once both are timed
        cudaEvent_t ev[4] = {};                   // graph launch and direct apply, start and end
    };
    GraphSlot graphs[3];                          // ewald_apply, ewald_apply_forces, ewald_apply_host
    bool graphs_off = false;                      // a capture failed: direct launches from then on
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev[ewg::kNumEvents] = {};
    int timing = 0;                               // 0 off, 1 timed, 2 timed with serialised stages
    bool timed_once = false;
    bool positions_valid = false;
    int64_t footprint = 0;
};

namespace ewg {

// ---- host-side math shared by the planner (no CUDA) ----------------------
double bessel_i0(double x);
double kb_window(double t_grid, int P);                  // w_0 at t (grid units)
double kb_window_hat(double k, double h, int P);          // closed-form transform
ewald_status fit_window(int P, int deg, WindowPoly *out, double *max_err);
ewald_status choose_params(int64_t N, double L, double tol, ewald_dtype dtype,
                           const ewald_params *ov, ewald_params *out);
// radius (length units) inside which a double-single plan's near-field pairs
// run in double-single, the rest in compensated FP32 (rc: all double-single)
double ds_split_radius(double tol, double xi, double rc);

// ---- kernel launchers (defined in the .cu files) -------------------------
struct BinArgs {
    const double *x;     // user positions N x 3
    const double *f;     // user forces N x 3 (may be null: positions only)
    int64_t N;
    double L, cell, h;
    int nc, M, P, T, nt;
    bool f64;            // sorted arrays in FP64 (else FP32)
    bool tf_ds;          // tile-sorted forces as double-single pairs of float4
};
cudaError_t launch_bin_keys(ewald_plan_s *p, const BinArgs &a, cudaStream_t s);
cudaError_t launch_scan(const int32_t *in, int32_t *out, int n, cudaStream_t s);
// binning's scans in one launch: sub-cell and tile starts, and the P2P work
// items per cell with their offsets
cudaError_t launch_bin_scans(ewald_plan_s *p, cudaStream_t s);
cudaError_t launch_bin_scatter(ewald_plan_s *p, const BinArgs &a, cudaStream_t s);
cudaError_t launch_gather_forces(ewald_plan_s *p, const double *f, cudaStream_t s);
cudaError_t launch_cell_items(ewald_plan_s *p, cudaStream_t s);  // the work items alone
cudaError_t launch_p2p(ewald_plan_s *p, cudaStream_t s);
cudaError_t launch_p2g(ewald_plan_s *p, cudaStream_t s);
// P2G of three tile-order source components `tfrc` (the plan's force layout)
// onto the 3-component grid `grid`
cudaError_t launch_p2g_with(ewald_plan_s *p, const void *tfrc, void *grid, cudaStream_t s);
// double layer (k_dl.cu)
cudaError_t launch_dl_densities(ewald_plan_s *p, const double *q, const double *n, cudaStream_t s);
cudaError_t launch_scale_dl(ewald_plan_s *p, double C, cudaStream_t s);
// FP32 plans (FP32 near field and FFTs): the double layer's near field on the
// Stokeslet P2P machinery -- 48-byte near-order source records (positions
// from the plan's FP32 records, S = sym(q (x) n)), then the sum into u
cudaError_t launch_dl_records(ewald_plan_s *p, const double *q, const double *n, void *drec, cudaStream_t s);
// P2G of the Stokeslet forces and the double layer's two density triples
// (dl_tf: 2 N float4 in tile order) in one pass onto p->grid and the two
// 3-component grids at dl_grid (FP32-kernel plans with 8^3 tiles)
bool p2g9_supported(const ewald_plan_s *p);
cudaError_t launch_p2g9(ewald_plan_s *p, const void *dl_tf, void *dl_grid, cudaStream_t s);
// adds the double layer's FP32 near field into p->un (FP32 plans: after the Stokeslet P2P, same stream)
cudaError_t launch_p2p_dl32(ewald_plan_s *p, const void *drec, cudaStream_t s);
cudaError_t launch_p2p_dl(ewald_plan_s *p, const double *x, const double *q, const double *n, double *u,
                          cudaStream_t s);
cudaError_t launch_scale(ewald_plan_s *p, double C, cudaStream_t s);
bool fgc_z_supported(int M);
cudaError_t launch_fgc_z(ewald_plan_s *p, double C, cudaStream_t s);
// the same with the double layer's six density spectra (dl_spec) added in the CNV
cudaError_t launch_fgc_z_dl(ewald_plan_s *p, double C, cudaStream_t s);
// FP64 spectra: the z transforms and the CNV in double-single arithmetic (k_fgc_z64.cu)
cudaError_t launch_fgc_z64(ewald_plan_s *p, double C, cudaStream_t s);
// FP64 spectra: the y transforms (forward or inverse) in double-single
// arithmetic, between cuFFT's 1-D transforms along x and the z kernel
cudaError_t launch_fft_y64(ewald_plan_s *p, bool inv, cudaStream_t s);
// G2P from a grid in the kernels' precision (FP64 when near64, else FP32; the
// double-single planes for grid_ds plans); the sum is multiplied by `scale`.
cudaError_t launch_g2p(ewald_plan_s *p, const void *grid, double scale, cudaStream_t s);
cudaError_t load_p2p_constants();
// The near field of many plans: one persistent launch per P2P variant over
// all their work items (the plans' own buffers; they must stay alive).
struct P2PBoxes;
cudaError_t p2p_boxes_create(ewald_plan_s *const *plans, int n, P2PBoxes **out);
cudaError_t p2p_boxes_launch(const P2PBoxes *b, cudaStream_t s);
int p2p_boxes_launches(const P2PBoxes *b);
void p2p_boxes_destroy(P2PBoxes *b);
// Batches: every box's binning, sum and FP64 -> FP32 grid copies as one
// launch per kernel (k_bin.cu); x, f, u per box are its batch buffers.
struct BinBoxes;
cudaError_t bin_boxes_create(ewald_plan_s *const *plans, const double *const *x, const double *const *f,
                             double *const *u, int n, BinBoxes **out);
cudaError_t bin_boxes_launch(const BinBoxes *b, cudaStream_t s);
cudaError_t sum_boxes_launch(const BinBoxes *b, cudaStream_t s);
int bin_boxes_launches(const BinBoxes *b);
int sum_boxes_launches(const BinBoxes *b);
void bin_boxes_destroy(BinBoxes *b);
struct ConvBoxes;
cudaError_t conv_boxes_create(const std::vector<const void *> &src, const std::vector<void *> &dst,
                              const std::vector<int64_t> &n, ConvBoxes **out);
cudaError_t conv_boxes_launch(const ConvBoxes *b, cudaStream_t s);
int conv_boxes_launches(const ConvBoxes *b);
void conv_boxes_destroy(ConvBoxes *b);
// P2G (kind 0) and G2P (kind 1) of many plans: one launch per kernel
// instantiation (k_grid.cu; plans with double-single grid kernels excluded)
struct GridBoxes;
cudaError_t grid_boxes_create(ewald_plan_s *const *plans, void *const *grid, void *const *g2p, int n, GridBoxes **out);
cudaError_t grid_boxes_launch(const GridBoxes *b, int kind, cudaStream_t s, int fft64);
int grid_boxes_launches(const GridBoxes *b);
void grid_boxes_destroy(GridBoxes *b);
// the double-single grid stages of many plans (k_grid_ds.cu): stage 0 window
// weights, 1 P2G, 2 the double-single grid copies, 3 G2P
struct DsGridBoxes;
cudaError_t ds_grid_boxes_create(ewald_plan_s *const *plans, double *const *grid, float *const *gds, int n,
                                 DsGridBoxes **out);
cudaError_t ds_grid_boxes_launch(const DsGridBoxes *b, int stage, cudaStream_t s);
int ds_grid_boxes_launches(const DsGridBoxes *b);
void ds_grid_boxes_destroy(DsGridBoxes *b);
// the CNV of many plans in one launch per precision (k_fgc.cu)
struct ScaleBoxes;
cudaError_t scale_boxes_create(ewald_plan_s *const *plans, void *const *spec, int n, ScaleBoxes **out);
cudaError_t scale_boxes_launch(const ScaleBoxes *b, cudaStream_t s, int fft64);
int scale_boxes_launches(const ScaleBoxes *b);
void scale_boxes_destroy(ScaleBoxes *b);
// Batches: the plan's real grid and half spectrum replaced by slices of a
// batch-owned buffer (its own are freed; the batch frees the new ones).
ewald_status plan_adopt_grid(ewald_plan_s *p, void *grid, void *spec);
cudaError_t launch_sum(ewald_plan_s *p, const double *f, double *u, cudaStream_t s);
// Recreate the plan's own streams (the near-field side stream and the graph
// capture origin) with a CUDA stream priority, for a server slot whose stream
// has that priority.  The plan must be idle.
ewald_status plan_set_stream_priority(ewald_plan_s *p, int priority);
cudaError_t launch_copy_out(const void *src, bool src_f64, double *dst, int64_t n, cudaStream_t s);
// Served requests: f <- f + a n (Philox4x32-10 normals for (point, step,
// seed)), then f <- f - mean(f); `sums` is 3 doubles of device scratch.
cudaError_t launch_perturb_forces(double *f, int64_t N, double a, uint32_t step, uint64_t seed,
                                  double *sums, cudaStream_t s);
cudaError_t launch_grid_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t n,
                                cudaStream_t s);
// Double-single grid kernels (k_grid_ds.cu): usable for tile 8, kGridDsMinP <=
// P <= kMaxP, M <= 1024.  The window weights of the tile-sorted points (after
// binning), P2G into the FP64 grid, G2P from a double-single copy of it (3 M^3
// h values then 3 M^3 l values), and that copy.
bool grid_ds_supported(int P, int T, int M);
// TMA descriptor of a planar FP32 grid [nc][M][M][M] with boxes of (x, y, z,
// c) = (S, RR, RR, bc) floats (k_grid.cu); false if it cannot be made
bool grid_tensor_map(const void *grid, int M, int nc, int S, int RR, int bc, struct CUtensorMap_st *m);
cudaError_t launch_window_ds(ewald_plan_s *p, cudaStream_t s);
cudaError_t launch_p2g_ds(ewald_plan_s *p, cudaStream_t s);
// P2G of three tile-order source components in the double-single force
// format ((h.xyz, 0), (l.xyz, 0) per point) onto the 3-component FP64 grid
cudaError_t launch_p2g_ds_with(ewald_plan_s *p, const void *tfrc, double *grid, cudaStream_t s);
cudaError_t launch_g2p_ds(ewald_plan_s *p, const float *gds, double scale, cudaStream_t s);
cudaError_t launch_grid_split(const double *src, float *dst, int64_t n, cudaStream_t s);

}  // namespace ewg
