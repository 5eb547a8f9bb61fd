// Host-side launch entry points of the CUDA kernels (one per kernel family).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernel_params.h"

namespace hvx {

// Persistent edge / Gaussian kernel over the tiles of many images.
struct EdgeBatchDesc {
    const CUtensorMap* maps;     // one per image, 64-byte aligned, in device memory
    const EdgeParams* params;    // one per image, in device memory
    const int* tile_start;       // n_img + 1 prefix sums of per-image tile counts
    const int* tiles_x;          // n_img tile columns per image (the kernel's tile width)
    int n_img;
    int total_tiles;
    int* err;
};

// Output mode of an edge / Gaussian group (which kernel instantiation runs it);
// every image of one batch launch must have the same mode.  EDGE_MODE_GAUSS
// (the Gaussian3x3 group alone) runs the Gaussian kernel, with its own tile;
// EDGE_MODE_BINOM5 (a 5x5 binomial Convolve alone) the binomial kernel, with
// the edge kernel's tiles and boxes.
constexpr int EDGE_MODE_GAUSS = 0;
constexpr int EDGE_MODE_BINOM5 = 7;
int edge_mode(const EdgeParams& p);
void edge_tile_dims(int mode, int* tw, int* th);
// output rows per thread of the single-image edge kernel for a W x H image
int edge_single_rows(int W, int H, int num_sms);
cudaError_t launch_edge(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s);
// rows: output rows per thread of the edge kernel's 128 x 8R tiles, R = 5,
// 10 or EDGE_ROWS (15, the default); the Gaussian kernel keeps its own tile
cudaError_t launch_edge_batch(const EdgeBatchDesc& d, int mode, int grid, cudaStream_t s,
                              int rows = EDGE_ROWS);
int edge_batch_blocks_per_sm(int mode);
// the fused edge kernel's Phase and mask arithmetic over every gradient pair
// in [-gmax, gmax]^2 ((2 gmax + 1)^2 bytes each, device memory)
cudaError_t launch_edge_point_selftest(int gmax, int s_thr, uint8_t* phase, uint8_t* mask,
                                       cudaStream_t s);

// one image; p.rows (2, 5 or GAUSS_ROWS) rows per thread, the map boxed
// 160 x (8 p.rows + 2)
cudaError_t launch_gauss(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s);
int gauss_single_rows(int W, int H, int num_sms);
cudaError_t launch_gauss_batch(const EdgeBatchDesc& d, int grid, cudaStream_t s);
int gauss_batch_blocks_per_sm();

// 5x5 binomial Convolve: one image (p.rows 2 or 5, the map boxed 160 x
// (8 p.rows + 4)), or a batch with 128 x 8 rows tiles (rows 5, 10, 15)
cudaError_t launch_binom5(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s);
cudaError_t launch_binom5_batch(const EdgeBatchDesc& d, int grid, int rows, cudaStream_t s);
int binom5_batch_blocks_per_sm();

// Harris: the UNDEFINED-border fast kernel or the general one; the tensor map
// of the group's input must use the box harris_box() gives.
bool harris_fast_path(const HarrisParams& p);
int harris_fast_rows(int W, int H, int num_sms);
void harris_box(const HarrisParams& p, int* w, int* h);
cudaError_t launch_harris(const CUtensorMap& map, const HarrisParams& p, cudaStream_t s);
// BORDER_UNDEFINED Harris over n images in one launch (every image's rows
// equal; tensor maps boxed for them); total = tile_start[n]; resp: some
// image exports its response
cudaError_t launch_harris_batch(const CUtensorMap* maps, const HarrisParams* ps,
                                const int* tile_start, const int* tiles_x, int n, int total,
                                bool tomasi, bool resp, cudaStream_t s);
int harris_fast_tile_w();
int harris_batch_rows(const int* W, const int* H, int n, int num_sms);
cudaError_t launch_generic(const GenericDesc& d, cudaStream_t s);
cudaError_t launch_plain(const PlainParams& p, cudaStream_t s);
cudaError_t launch_eqhist(const EqHistParams& p, cudaStream_t s);

}  // namespace hvx
