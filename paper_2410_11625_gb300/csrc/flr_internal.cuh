// flr_internal.cuh -- definitions shared by the FLR kernels and the C ABI layer of
// libflr.so (not installed; the public interface is include/flr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "flr.h"

namespace flr {

// ---- moment channels ---------------------------------------------------------------
//
// The window sums FLR needs per pixel (Sec. 3.2 box-filters the outer products of the
// guide vector with its leading 1, x x^T, and of x with the radiance, x y^T):
//   sum x_i        (Q)      linear guide moments         -> mu_X * n   (Appendix u_X)
//   sum y_c        (3)      linear radiance moments      -> mu_Y * n
//   sum x_i x_j    (Q(Q+1)/2, i <= j)                    -> S
//   sum x_i y_c    (3Q)                                  -> X^T Y without its top row
// n itself is the number of in-image pixels of the clipped window and is computed from
// the geometry.  Channels are numbered in the order above.
template <int Q>
struct Chan {
    static constexpr int NX = Q;
    static constexpr int NY = 3;
    static constexpr int NXX = Q * (Q + 1) / 2;
    static constexpr int NXY = 3 * Q;
    static constexpr int NCH = NX + NY + NXX + NXY;
    static constexpr int X0 = 0;
    static constexpr int Y0 = Q;
    static constexpr int XX0 = Q + 3;
    static constexpr int XY0 = Q + 3 + NXX;
    static constexpr int NSLOT = Q + 3;  // input slots: Q guides then 3 radiance channels

    __host__ __device__ static constexpr int xx(int i, int j)
    {  // i <= j, upper triangle row by row
        return XX0 + i * Q - (i * (i - 1)) / 2 + (j - i);
    }
    __host__ __device__ static constexpr int xy(int i, int c) { return XY0 + 3 * i + c; }

    // Input slots multiplied to form channel ch (second = -1 for a linear channel).
    __host__ __device__ static constexpr int slot_u(int ch)
    {
        if (ch < XX0) return ch;  // x_i or y_c
        if (ch < XY0) {
            int k = ch - XX0, i = 0;
            while (k >= Q - i) { k -= Q - i; ++i; }
            return i;
        }
        return (ch - XY0) / 3;
    }
    __host__ __device__ static constexpr int slot_v(int ch)
    {
        if (ch < XX0) return -1;
        if (ch < XY0) {
            int k = ch - XX0, i = 0;
            while (k >= Q - i) { k -= Q - i; ++i; }
            return i + k;
        }
        return Q + (ch - XY0) % 3;
    }

    // The vertical-sum walkers of the forward kernel split the channels into three
    // contiguous groups of similar size: [0, G1) = linear moments and the first rows of
    // the x x^T triangle, [G1, XY0) = the remaining rows, [XY0, NCH) = x y^T.
    __host__ __device__ static constexpr int rows_upto(int i1)
    {
        int s = 0;
        for (int i = 0; i < i1; ++i) s += Q - i;
        return s;
    }
    __host__ __device__ static constexpr int split_row()
    {
        int best = 0, best_cost = 1 << 30;
        for (int i1 = 0; i1 <= Q; ++i1) {
            int g0 = XX0 + rows_upto(i1), g1 = NXX - rows_upto(i1);
            int cost = g0 > g1 ? g0 : g1;
            if (cost < best_cost) { best_cost = cost; best = i1; }
        }
        return best;
    }
    static constexpr int G1 = XX0 + rows_upto(split_row());
    __host__ __device__ static constexpr int group_begin(int g) { return g == 0 ? 0 : (g == 1 ? G1 : XY0); }
    __host__ __device__ static constexpr int group_end(int g) { return g == 0 ? G1 : (g == 1 ? XY0 : NCH); }
    __host__ __device__ static constexpr int group_size(int g) { return group_end(g) - group_begin(g); }
    __host__ __device__ static constexpr int max_group()
    {
        int m = 0;
        for (int g = 0; g < 3; ++g) m = group_size(g) > m ? group_size(g) : m;
        return m;
    }
    static constexpr int GMAX = max_group();
};

// ---- launch geometry of the forward kernel ----------------------------------------------
constexpr int kTW = 96;        // output columns of one strip
constexpr int kB = 4;          // rows solved per batch
constexpr int kThreads = 384;  // = kB * kTW: one solver thread per pixel of a batch
static_assert(kB * kTW == kThreads, "one solver thread per batch pixel");
constexpr int kShiftSamples = 16;  // the shifts are means over a 16 x 16 sample grid

struct FwdArgs {
    const float *guide, *map_guide, *rad;
    float *out;   // [3][H][W] written when rc == 0
    float *coef;  // [(Q+1)*3][H][W] per-pixel models written when rc > 0
    int H, W, r, rc;
    float eps, tau;
    int TH;                          // rows per segment (a multiple of kB)
    unsigned long long *flag_count;  // device counter of flagged pixels
    int *flag_list;                  // flagged pixel indices y * W + x
    int flag_cap;
    float *shift_out;  // frame reference shift (Q+3 floats), written by block (0, 0)
    int force_coef;    // write the coefficient planes even when rc == 0 (backward pass)
    // adjoint mode only: G(A_k) planes in, per-pixel moment gradients out, d/d eps
    const float *gA;   // [(Q+1)*3][H][W]: row 0 = G(b_k), rows 1..Q = G(a_k)
    float *gS;         // [NCH][H][W] in moment-channel order (see Chan)
    double *geps;      // accumulated d L / d eps
    int *status = nullptr;  // set to 1 if a bounded device wait ran out (may be NULL)
    unsigned long long *nonfinite = nullptr;  // count of non-finite output values (may be NULL)
    // rows [row_lo, row_hi) of the frame are computed (row_hi < 0: to H); the frame reference
    // is sampled over rows [0, ref_rows) (ref_rows <= 0: all rows)
    int row_lo = 0, row_hi = -1, ref_rows = 0;
};

struct ApplyArgs {
    const float *coef, *map_guide, *shift;
    float *out;
    int H, W, rc;
    int *status = nullptr;  // set to 1 if a bounded device wait ran out (may be NULL)
    int row_lo = 0, row_hi = -1;  // output rows [row_lo, row_hi) (row_hi < 0: to H)
    unsigned long long *nonfinite = nullptr;  // count of non-finite output values (may be NULL)
};

struct Fp64Args {
    const float *guide, *map_guide, *rad, *shift;
    float *out, *coef;
    int H, W, r, rc;
    int force_coef;  // write the model to the coefficient planes even when rc == 0
    double eps;
    const unsigned long long *flag_count;
    const int *flag_list;
    int flag_cap;
    const unsigned long long *flag_start = nullptr;  // first list entry to re-solve (NULL: 0)
    unsigned long long *nonfinite = nullptr;  // count of non-finite output values (may be NULL)
};

struct BwdArgs {
    const float *guide, *rad, *shift, *g;  // inputs, frame reference shift, dL/dI
    const float *BS;                       // [NCH] box-summed moment gradients
    const float *BA;                       // [(Q+1)*3] box-summed (rc > 0) or raw models
    float *grad_guide, *grad_map, *grad_rad;
    int H, W, rc;
    int separate_map;                      // the map guide is not the model guide
};

// Arguments of the fused forward kernel (flr_fused.cu) and of its FP64 correction kernel.
struct FusedArgs {
    const float *guide, *map_guide, *rad;
    float *out;
    int H, W, r, rc;
    float eps, tau;
    int TH;                          // output rows per segment (grid.y segments)
    int row_lo = 0, row_hi = -1;     // output rows [row_lo, row_hi) (row_hi < 0: to H)
    int *list;                       // flagged pixels: CTA c's entries at list + c * list_cap
    int list_cap;                    // >= the pixels one CTA solves, (TW + 2 rc) (TH + 2 rc)
    int *list_count;                 // entries per CTA, written by every CTA of the launch
    float *cta_shift;                // per CTA: its reference shift, Q + 3 floats
    unsigned long long *flag_count = nullptr;  // flagged pixels owned by a CTA (fix kernel)
    unsigned long long *nonfinite = nullptr;   // non-finite output values (may be NULL)
    int *status = nullptr;                     // set to 1 if a bounded wait ran out (may be NULL)
};

// Host-side plan and checks shared by the entry points of flr_capi.cu and flr_noalloc.cu
// (defined in flr_capi.cu).
namespace host {
int validate_params(const flr_params *p);
int choose_segment_rows(int H, int W, int r, int n_sm);
// Launch plan of the fused forward kernel over `rows` output rows: strips of TW columns and
// segments of TH rows; cap = pixels one CTA solves, (TW + 2 rc)(TH + 2 rc).
struct FusedPlan {
    int TW, TH, strips, segs, cap;
};
FusedPlan fused_plan(int rows, int W, int r, int rc, int n_sm);
bool fused_ok(const flr_params &p, int H, int W, const void *g, const void *mg, const void *rad, const void *out);
}  // namespace host

// Host-side launchers (defined in the .cu files; q is dispatched to a template).
bool fused_supported(int q, int r, int rc);
int fused_tile_width(int rc);
cudaError_t launch_fused(int q, const FusedArgs &a, dim3 grid, cudaStream_t st);
cudaError_t launch_fused_fix(int q, const FusedArgs &a, dim3 grid, cudaStream_t st);
cudaError_t launch_fwd(int q, const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st);
cudaError_t launch_adj(int q, const FwdArgs &a, dim3 grid, size_t smem, cudaStream_t st);
cudaError_t adj_prepare(int q, int r, size_t smem);
size_t fwd_smem_bytes(int q, int r);
size_t adj_smem_bytes(int q, int r);
cudaError_t fwd_prepare(int q, int r, size_t smem);
cudaError_t launch_apply(int q, const ApplyArgs &a, cudaStream_t st);
cudaError_t launch_fp64(int q, const Fp64Args &a, int n_sm, cudaStream_t st);
cudaError_t launch_bwd_fields(int q, const float *g, const float *z, const float *shift, float *F, int H, int W,
                              int rc, cudaStream_t st);
cudaError_t launch_box_sum(const float *in, float *out, int nplanes, int H, int W, int rad, cudaStream_t st,
                           int *status = nullptr);
cudaError_t launch_bwd_contract(int q, const BwdArgs &a, cudaStream_t st);
// the frame reference shift of the forward kernel (Q + 3 floats), by itself
cudaError_t launch_frame_shift(int q, const float *guide, const float *rad, int H, int W, int ref_rows, float *shift_out,
                               cudaStream_t st);
namespace fast { struct FastArgs; }
bool batch_supported(int q, int F);
cudaError_t launch_batch(int q, int F, const void *args, cudaStream_t st);
size_t batch_args_size();
void fill_batch_args(void *args, int n, const fast::FastArgs *frames, unsigned *count, unsigned *gen, int *status);
cudaError_t launch_barrier_selftest(unsigned *count, unsigned *gen, unsigned expected, int *status,
                                    unsigned long long timeout_ns, int grid, cudaStream_t st);

}  // namespace flr
