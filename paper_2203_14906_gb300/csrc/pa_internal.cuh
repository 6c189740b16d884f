// pa_internal.cuh -- types shared by the kernels and the host plan code of
// the HO-DMAS beamformer (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_hodmas.h"

namespace pa {

// Columns handled by one thread.  The thread's pixels sit at columns
// jt, jt+m, ..., jt+(kC-1)m of one depth row, so at channel step u they all
// need the delay of the same lattice offset d = jt - m*u (pixel c pairs with
// channel i = u + c): one table load serves kC pairs.
constexpr int kC = 4;
// Channel steps per shared-memory chunk (chosen per plan, a multiple of kC,
// at most kNCMax) and the virtual channels staged per chunk (steps + kC - 1).
constexpr int kNCMax = 72;
constexpr int kNCSMax = kNCMax + kC - 1;
// Channel steps between Kahan folds of the compensated power sums: plain
// FP32 partial sums over 64 channels, compensated across folds.  Every fold
// loads and stores each accumulator's totals in TMEM (about 100 instructions
// per thread), so its issue cost per pair halves with the interval.
// Measured on GB300 (BF16 RF, 128 channels, k = 3, 32 frames, fused kernel
// per launch): folding every 8 / 16 / 32 steps took 0.937 / 0.894 / 0.877 ms
// in an earlier build with the totals in registers; with the totals in TMEM
// every 32 / 64 steps takes 0.676 / 0.661 ms (cfg3, 256 channels: k = 3
// 1.289 / 1.259 ms, k = 5 1.586 / 1.547 ms).
constexpr int kFoldBlocks = 16;  // blocks of kC steps
constexpr int kMaxOrder = 8;
// Shared-memory layout of the fused kernel: work-item words, the TMA
// mbarrier (8 B at 16) and the TMEM base address (4 B at 24), channel bases
// and window starts (kCbInts ints each,
// >= kNCSMax + 1, multiple of 4), the raw TMA buffer (128-byte aligned, empty
// without TMA), then the interpolation slots.
constexpr int kCbInts = 76;
constexpr int kMbarOff = 16;
constexpr int kTmemOff = 24;
constexpr int kCbOff = 32;
constexpr int kLoOff = kCbOff + kCbInts * 4;
constexpr int kRawOff = 640;  // >= kLoOff + 4 kCbInts, 128-byte aligned
static_assert(kRawOff >= kLoOff + kCbInts * 4 && kRawOff % 128 == 0, "shared layout");
constexpr int kMaxThreads = 1024;

// TMEM columns a fused-kernel block allocates for compensated totals (a
// power of two >= 32): the warps sharing a 32-lane quarter of TMEM times 8
// columns per accumulator (kC totals and kC compensation terms).
__host__ __device__ constexpr int tmem_columns(int warps, int na) {
  return ((warps + 3) / 4) * na * 8 <= 32    ? 32
         : ((warps + 3) / 4) * na * 8 <= 64  ? 64
         : ((warps + 3) / 4) * na * 8 <= 128 ? 128
                                              : 256;
}
// TMEM columns of one SM.
constexpr int kTmemColsPerSm = 512;

// Delay-table layout, row t = d - dmin (lattice offset d), depth z:
// zb = 0: row-major, depth fastest (nzp entries per row);
// zb > 0: depth blocks of 2^zb rows, within a block row-major.  With 8-row
// lane groups and zb = 3 a warp's step loads (8 depth rows of 4 neighbouring
// lattice rows) are one contiguous 256-byte run instead of four 64-byte
// pieces.
__host__ __device__ __forceinline__ size_t table_index(int t, int z, int ndrows, int nzp, int zb) {
  if (zb == 0) return (size_t)t * nzp + z;
  return (((size_t)(z >> zb) * ndrows + t) << zb) + (z & ((1 << zb) - 1));
}

// Parameters of the fused gather + interpolate + root + power-sum kernel.
struct BfParams {  // aligned as CUtensorMap requires
  CUtensorMap tmap;       // 3-D RF map [frames][N][Ns], box {wr, 1, 1} (TMA path)
  int use_tma;            // 1: stage with TMA boxes, 0: vectorised loads
  int wr;                 // raw samples per channel delivered by one TMA box
  int rp;                 // row pitch of the raw buffer in samples (128-byte rows)
  int chunk_bytes;        // bytes one chunk's TMA boxes deliver
  int pairs_off;          // byte offset of the interpolation slots
  const void* rf;         // [frames][N][Ns] in rf_dtype
  int rf_dtype;           // pa_rf_dtype
  int vec_ok;             // rows start 8/16-byte aligned (Ns % 4 == 0)
  int nearest;            // 1: nearest-sample delays (a = 0), one tap per pair
  int lane_rows_log2;     // log2 of the depth rows per lane group: 5, 4 or 3
  int nc, ncs;            // channel steps per chunk, virtual channels staged per chunk
  int tmem_cols;          // TMEM columns a block allocates (compensated sums), else 0
  int n_elem, n_samples;
  long long frame_elems;  // N * Ns
  const int2* table;      // lattice table [ndrows][nz_pad] {n0 * 8, float bits of a},
                          // rows = lattice offsets
  const int2* ftab;       // full table, in the kernel's read order: per tile,
                          // channel step (steps + 3), pixel half c / 2, thread
                          // of the tile, pixel c % 2: {(n0 - window start) * 8,
                          // float bits of a}
  int full;               // 1: full table (channel bases are window starts)
  int steps;              // channel steps u1 - u0
  const float* wtab;      // [ndrows][nz_pad] apodisation weight (or null)
  int table_stride;       // entries between lattice rows at one depth (nz_pad or 2^zb)
  const int4* items;      // [n_tiles * ngroups] {tile_id, grp, tx, tz}, deepest first
  const int2* slot_rg;    // [slots] {column residue r_m, column group g}
  int ndrows;
  int dmin;               // lattice offset of table row 0
  int m;                  // column stride of a thread's pixels (lattice: pitch / dx)
  int R;                  // column groups per residue in a tile
  int nxt, nzt;           // tiles along x and z
  int tile_x, tile_z;
  int warps;              // warps per block
  int slots;              // warp slots per tile (m * R)
  int ngroups;            // residue groups per tile (slots / warps)
  int nv;                 // virtual channels (zero rows pad both ends)
  int u0;                 // first channel step (= -(kC-1))
  int window;             // float2 slots staged per channel (multiple of 4)
  int w4_inv;             // ceil(2^20 / (window / 4)): exact idx / (window / 4) by multiply-shift
  const int* lo;          // [n_tiles][nv] first staged sample per channel
  const int2* urange;     // [n_tiles][warps] channel-step range of a warp
  const int2* vchunks;    // [n_tiles] chunk range of a tile
  float* out;             // output base
  int planes;             // planes per frame (n_stages * n_outputs)
  int plane_das, plane_dmas, plane_ho;  // raw plane of each output or -1
  int nx, nz;
  int n_frames;           // frames in this launch
  int n_items;            // n_tiles * n_frames
  int* counter;           // work counter (zeroed before launch)
  int* err;               // error flags: 1, 2 index checks (checked builds), 8 a wait ran out
  int* timeouts;          // running count of blocks whose bounded TMA wait ran out
  int expect_extra;       // bytes added to every chunk's expected transaction
                          // count: 0, or > 0 only to test the bounded wait
  // entry of table row 0 at depth z: (z >> table_zshift) * table_zblock +
  // (z & table_zmask) (row-major: shift 31, block 0, all-ones mask)
  int table_zshift, table_zmask;
  long long table_zblock;
  int table_zb, table_nzp;  // the layout for table_index (zb 0: row-major)
};

// Post-filter / envelope parameters (one warp per depth column).
struct PostParams {
  float* out;
  int planes;          // planes per frame
  int n_out;           // outputs per stage
  int s_src, s_dst;    // stage index holding raw / receiving the envelope
  int nx, nz, m, log2m;
  const float2* tw;    // per-pass twiddle blocks (see twiddles() in pa_post.cu)
  int n_tw;            // entries of tw
  const float* mask;   // [n_out][m] band-pass x analytic mask
  int* maxslot;        // [frames][n_out] float bits of the image maximum
  int n_frames;
  int warps_per_block;
};

struct LogParams {
  float* out;
  int planes, n_out, s_src, s_dst;
  long long plane_elems;  // nx * nz
  const int* maxslot;
  float dyn_range_db;
  int n_frames;
};

// A kernel launch described as data (direct launch or CUDA-graph node).
struct LaunchSpec {
  const void* func = nullptr;
  dim3 grid, block;
  size_t smem = 0;
};

const void* bf_func(int order, bool apod, bool comp, bool full);
void post_spec(const PostParams& p, LaunchSpec* s);
// Radix of the first FFT pass of the in-place post kernel (the passes after
// it are radix 8, then one radix-4 or radix-2 pass for the remainder); the
// host builds the per-pass twiddle tables in the same order.
__host__ __device__ constexpr int post_first_radix(int m) { return m == 1024 ? 16 : 8; }
// Post-kernel buffers keep one padding slot every 2^post_pad_shift(M)
// complex elements (16 from 256 points on, else 8).
__host__ __device__ constexpr int post_pad_shift(int m) { return m >= 256 ? 4 : 3; }
__host__ __device__ constexpr int post_padded_len(int m) { return m + (m >> post_pad_shift(m)); }
int post_buffers(int m);     // M-point complex buffers per team of the post kernel
const void* post_inplace_func(int m);  // in-place kernel for M points, or nullptr
int post_team_warps(int m);  // warps per team (column pair) of the post kernel
void log_spec(const LogParams& p, int num_sms, LaunchSpec* s);

// Launchers (one translation unit per order keeps the builds parallel).
cudaError_t bf_launch(int order, bool apod, bool comp, bool full, const BfParams& p,
                      int grid, int block, size_t smem, cudaStream_t s);
cudaError_t bf_occupancy(int order, bool apod, bool comp, bool full, int block,
                         size_t smem, int* blocks_per_sm);

#define PA_DECLARE_ORDER(K)                                                 \
  cudaError_t bf_launch_k##K(bool apod, bool comp, bool full,               \
                             const BfParams& p, int grid, int block,        \
                             size_t smem, cudaStream_t s);                  \
  cudaError_t bf_occupancy_k##K(bool apod, bool comp, bool full, int block, \
                                size_t smem, int* blocks_per_sm);           \
  const void* bf_func_k##K(bool apod, bool comp, bool full);
PA_DECLARE_ORDER(1)
PA_DECLARE_ORDER(2)
PA_DECLARE_ORDER(3)
PA_DECLARE_ORDER(4)
PA_DECLARE_ORDER(5)
PA_DECLARE_ORDER(6)
PA_DECLARE_ORDER(7)
PA_DECLARE_ORDER(8)
#undef PA_DECLARE_ORDER

// Sets the thread-local message returned by pa_last_error().
void set_error_message(const char* msg);
// Device address of the plan's running count of timed-out waits (the word
// pa_beamform's launches update), for the server's completion check.
int* plan_timeout_counter(pa_plan_s* P);
// Device memory the plan owns (without synchronising, unlike pa_plan_get_info).
size_t plan_device_bytes(const pa_plan_s* P);
// The fused kernel's parameters for one launch of nf frames (what pa_beamform
// would launch), the plan's order, and whether the plan is the plain FP32
// lattice form with linear interpolation.
pa_status plan_bf_params(pa_plan_s* P, const void* rf, int nf, float* out, uint32_t stages,
                         BfParams* b, int* k, bool* lattice_fp32_plain);
// TMEM columns per fused-kernel block and whether the plan is TMEM-dense
// (its blocks can hold more TMEM than their register share of an SM).
void plan_tmem(const pa_plan_s* P, int* cols, bool* dense);

cudaError_t post_configure(size_t smem);
cudaError_t post_launch(const PostParams& p, cudaStream_t s);
cudaError_t log_launch(const LogParams& p, int num_sms, cudaStream_t s);

}  // namespace pa
