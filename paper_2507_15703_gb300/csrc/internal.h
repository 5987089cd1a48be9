// Internal interface between the host library (plan.cpp) and the CUDA kernel
// launchers (*.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cmb3d {

// Set the message cmb3d_error_detail() returns on this host thread (entry
// points outside plan.cpp use it to report why a call was rejected).
void set_error_detail(const char* msg);

// Packed half-spectrum buffer: float2 [N][N][N/2]; entry m_x' = 0 holds
// T(0,.,.) + i T(N/2,.,.).  After the three passes it holds float [N][N][N].

// Draw the Gaussian Fourier coefficients of realization key and inverse-FFT
// every (m_y, m_x') column along z.  amp[q] = sqrt(P_box(q) / 2) for
// q = m_x^2 + m_y^2 + m_z^2; tw[m] = exp(+2 pi i m / N), m < N.
// Kernel shape variants: v in [0, num_*_variants(N)); variant 0 is the default.
int num_col_variants(int N);
int num_draw_variants(int N);   // draw+z shapes: the column-pass shapes, then draw-only ones
int num_row_variants(int N);
int num_fused_variants(int N);

// key_dev != NULL: read the Philox key (seed lo, seed hi) from device memory.
// Only output z-planes in [zlo, zhi) are stored (zhi = 0: N), and with zmask
// != NULL (N bits) only those whose bit is also set.
cudaError_t launch_draw_zfft(int N, int v, float2* buf, const float* amp, const float2* tw,
                             uint64_t seed, cudaStream_t s, const uint2* key_dev = nullptr,
                             const uint32_t* zmask = nullptr, int zlo = 0, int zhi = 0, unsigned* err = nullptr);

// The draw with the z-transform as two 32-point split-FP16 DFT-GEMMs on the
// tensor cores (N = 1024; draw variant num_draw_variants(N) - 1).  *err is set
// if an MMA-completion wait gave up; err must not be NULL.
bool draw_tc_supported(int N);
cudaError_t launch_draw_tc(int N, float2* buf, const float* amp, const float2* tw, uint64_t seed, cudaStream_t s,
                           unsigned* err, const uint2* key_dev = nullptr, const uint32_t* zmask = nullptr,
                           int zlo = 0, int zhi = 0);

// 2-D Fourier method: the hybrid layers [z][m_y][m_x'] (h <= 32 layers) from
// the per-q table of z-covariance square roots (h x h floats per q).
cudaError_t launch_draw2d(int N, int h, float2* buf, const float* tab, uint64_t seed, cudaStream_t s);

// Diagnostic: the drawn packed half spectrum [m_z][m_y][m_x'], untransformed.
cudaError_t launch_draw_only(int N, float2* buf, const float* amp, uint64_t seed, cudaStream_t s);

// Inverse FFT of every (z, m_x') column along y, in place.
// With `planes` only the nplanes listed z-planes are transformed, and with
// `rowmask` (N bits per z-plane, bit y of word z N/32 + y/32) only the marked
// rows of them are stored.
cudaError_t launch_yfft(int N, int v, float2* buf, const float2* tw, cudaStream_t s, const int32_t* planes = nullptr,
                        int nplanes = 0, const uint32_t* rowmask = nullptr);

// Fused y and x passes (one thread-block cluster per z-plane, the plane kept in
// L2 between the two axes, or for variant 2 at N = 256, 512 in the cluster's
// distributed shared memory); num_fused_variants(N) > 0 for 128 <= N <= 1024.
cudaError_t launch_yx_fused(int N, int v, float2* buf, const float2* tw, cudaStream_t s);
// Whether fused variant v can run on the current device (cluster shape fits).
bool fused_variant_available(int N, int v);

// FFT along y with the radix-16 stages as split-FP16 DFT-GEMMs on the tensor
// cores (N = 256, 512, 1024).  *err is set if an MMA-completion wait gave up.
bool yfft_gemm_supported(int N);
cudaError_t launch_yfft_gemm(int N, float2* buf, const float2* tw, unsigned* err, cudaStream_t s);

// Complex-to-real inverse FFT of every (z, y) row along x, in place.
// With `rows` (row indices z N + y, nrows a multiple of the shape's rows per
// block: kRowListPad covers every shape for N >= 128, kRowListPadAny every N)
// only the listed rows are transformed; padding entries must name a scratch row.
constexpr int ilog2i(int n) { return n <= 1 ? 0 : 1 + ilog2i(n >> 1); }
constexpr int kRowListPad = 64;
constexpr int kRowListPadAny = 256;
// With `cols` (one word per listed row) the transformed row is stored only in
// the column blocks whose bit is set, block b holding columns [b N/32, (b+1) N/32):
// the blocks the interpolation stencils of a sky map read.
cudaError_t launch_xc2r(int N, int v, float2* buf, const float2* tw, cudaStream_t s, const int32_t* rows = nullptr,
                        int64_t nrows = 0, const uint32_t* cols = nullptr);

// Interpolate the field float[z][y][x] at npix pixels.  tab[i] = (tx, ty, tz,
// packed base cell) in gather order; out[perm[i]] receives pixel i (perm may
// be NULL for the identity).
// The x pass fused with the gather.  Pixels are grouped at plan time by the
// kXgTile x kXgTile tile of (z, y) base cells they fall in; an entry is one
// tile (or, where a tile's stencils reach more than kXgCols distinct x, a
// part of it split by x).  Its block transforms the (z, y) rows the entry's
// stencils read into a shared patch [slot][column] holding only the entry's
// needed x columns, then interpolates its pixels from the patch with the
// arithmetic of interpolate() (gather_tiles.cuh).  Row slot = lz S + ly for
// local offsets lz, ly in [0, S), S = kXgTile + K - 1 (K taps per axis), at
// global z = (z0 + lz + OFF) mod N (likewise y); padded slots are -1 and read
// the scratch row.  The maps equal the separate x pass and gather bit for bit.
constexpr int kXgTile = 8;
constexpr int kXgCols = 64;
struct XgEntry {
  int32_t pix_begin, pix_end;    // pixels [pix_begin, pix_end) of the fused table
  int32_t row_begin, nrows;      // rows [row_begin, row_begin + nrows) of the slot and row lists
  int32_t col_begin, ncols;      // needed x columns, increasing
  int32_t z0, y0;                // tile origin in base cells
};
int xgather_rows_per_block(int N);                    // rows per batch; row lists are padded to it
bool xgather_supported(int N);
cudaError_t launch_xgather(int N, int interp, const float2* buf, const float2* tw, const XgEntry* entries,
                           int nentries, const int32_t* row_slot, const int32_t* row_glob, const int16_t* cols,
                           const float4* tab, const int32_t* perm, float* out, cudaStream_t s);

// With `runs` (a table sorted by base cell): runs[k] = (first pixel, count) of
// at most kGatherRun consecutive pixels sharing one base cell; each run's
// stencil is loaded once and every pixel of the run interpolated from it, with
// the arithmetic of the one-pixel form (maps bit for bit equal).
constexpr int kGatherRun = 8;
cudaError_t launch_gather(int N, int interp, const float* field, const float4* tab,
                          const int32_t* perm, float* out, int64_t npix, cudaStream_t s,
                          const int2* runs = nullptr, int64_t nruns = 0);

// ---- persistent batch kernel (batch.cu) ----------------------------------
struct BatchBox {
  float2* buf;            // the box's packed spectrum / field
  const float* amp;       // its amplitude table
  const float4* tab;      // its pixel table (gather order)
  const int32_t* perm;    // gather order -> caller order, or NULL
  float* out;             // caller's output
  int npix;
  uint32_t key_lo, key_hi;
  // the box's pruned transform (all NULL / whole ranges for a whole box)
  const int32_t* planes;  // z-planes the y pass transforms, or NULL for all N
  const uint32_t* rowmask;  // N bits per z-plane: rows the y pass stores, or NULL
  const int32_t* rows;    // (z, y) rows the x pass transforms, or NULL for all N^2
  const uint32_t* cols;   // per listed row, the column blocks to store (see launch_xc2r), or NULL
  const uint32_t* zmask;  // draw: N bits, planes to store when they are not one range, or NULL
  int zlo, zhi;           // draw: store the planes zlo <= z < zhi (without zmask)
  int ny_tiles, nx_blocks;  // y column tiles and x row blocks of this box
  unsigned nY, nX;        // its Y and X items (what its X and G items wait for)
};
enum { kBatchDraw = 0, kBatchY = 1, kBatchX = 2, kBatchG = 3 };
constexpr int kBatchTilesPerItem = 4;
constexpr int kBatchPixelsPerItem = 4096;
// Work item: box << 40 | type << 32 | index within (box, type).
inline uint64_t batch_item(int box, int type, int idx) {
  return (static_cast<uint64_t>(box) << 40) | (static_cast<uint64_t>(type) << 32) | static_cast<uint32_t>(idx);
}
bool batch_supported(int N);
// D items of a box, and the y tiles, x row blocks and Y, X items of a box
// whose y pass covers `nplanes` z-planes and x pass `nrows` rows (a multiple of
// kRowListPad, or N^2 for the whole box).
int batch_draw_items(int N);
void batch_box_counts(int N, int64_t nplanes, int64_t nrows, int* ny_tiles, int* nx_blocks, int* nY, int* nX);
int num_batch_variants();
cudaError_t batch_grid(int N, int interp, int v, int* blocks);
// ctr: [0] next item, [1] error word, [2 + 4 b + type] items of (b, type) done.
cudaError_t launch_batch(int N, int interp, int v, int grid, const BatchBox* boxes, const uint64_t* items,
                         int nitems, unsigned* ctr, const float2* tw, unsigned spin_limit, int withhold,
                         cudaStream_t s);

// Philox4x32-10 words of n counters (uint4 each).
cudaError_t launch_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                          cudaStream_t s);

// Packing of a pixel's base cell (bx, by, bz), each < 2048, into the fourth
// word of its table entry: bx | by << 11 | (bz & 1023) << 22, with bit 10 of bz
// carried in the sign bit of tz (tz >= 0).
inline uint32_t pack_cell(uint32_t bx, uint32_t by, uint32_t bz) {
  return bx | (by << 11) | ((bz & 1023u) << 22);
}

}  // namespace cmb3d
