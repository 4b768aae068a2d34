// Parameter block of the velocity network during training and the BF16
// operand images of the fused tensor-core training step (train_fused.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gmc {

// parameter block offsets (floats): W1 [256][32] (columns 25..31 zero), b1,
// W2, b2, W3, b3, W4, b4 ([256][256], [256]), W5 [4][256], b5 [4]
constexpr int64_t P_W1 = 0, P_B1 = 8192, P_W2 = P_B1 + 256, P_B2 = P_W2 + 65536,
                  P_W3 = P_B2 + 256, P_B3 = P_W3 + 65536, P_W4 = P_B3 + 256,
                  P_B4 = P_W4 + 65536, P_W5 = P_B4 + 256, P_B5 = P_W5 + 1024,
                  P_TOTAL = P_B5 + 4;
// the residual-modulated network continues the block with its condition
// shifts M_j [256][5] and channel scales G_j [2][256] of hidden layers 2-4
constexpr int64_t P_RM_M = P_TOTAL, P_RM_G = P_RM_M + 3 * 256 * 5,
                  P_TOTAL_RM = P_RM_G + 3 * 2 * 256;

// Standardization of the training data: condition and target means and
// inverse standard deviations (the sixth condition entry: the aspect of a
// network for rectangular cells, trained on the FP32 path).
struct Std {
  float cm[6], cis[6], ym[4], yis[4];
};

constexpr uint32_t kTagTrain = 6u;  // Philox tag of the batch draws

namespace tf {

// Batch rows drawn inside the forward kernel (Eq. 9): for row b of step k,
// Philox (seed, k B + b, event 0, kTagTrain) gives the sample index and t,
// event 1 the four normals x0; X0 = [cn, (1 - t) x0 + t x1, emb(t), 0],
// U = x1 - x0 (cn and x1 standardized).
struct Gen {
  const float *cond, *y;  // [5][n], [4][n]
  int64_t n;
  Std sd;
  uint64_t seed;
  int64_t step;
};

// Weight images (bytes; chunks of 64 K values, 128 B per row):
//   WF1      W1 as rows = 256 outputs, K = 32 inputs (one chunk, K 32..63 zero)
//   WF2..4   W_l as rows = outputs, K = inputs: 4 chunks of 256 rows (32 KB)
//   WF5      W5 as rows = 4 outputs (16 rows, 12 zero), K = inputs: 4 x 2 KB
//   WB5      W5^T as rows = 256 inputs, K = 4 outputs (K 4..63 zero)
//   WB4..2   W_l^T as rows = inputs, K = outputs: 4 chunks of 32 KB
constexpr uint32_t WF1 = 0, WF2 = 32768, WF3 = WF2 + 131072, WF4 = WF3 + 131072,
                   WF5 = WF4 + 131072, WB5 = WF5 + 8192, WB4 = WB5 + 32768,
                   WB3 = WB4 + 131072, WB2 = WB3 + 131072, WIMG_BYTES = WB2 + 131072;

// Per 128-row batch tile (bytes): X0^T (32 rows x 128 rows of K, two
// chunks), A_l^T and dZ_l^T (256 rows, two chunks of 32 KB), S_l (BF16
// pairs: word [channel pair][row]), dV (rows = batch, K = 4 outputs of 16),
// dV^T (16 rows, 4 used, two chunks of 2 KB).
constexpr uint32_t TILE_XT = 8192, TILE_AT = 65536, TILE_S = 65536, TILE_DV = 16384,
                   TILE_DVT = 4096;
constexpr uint32_t TILE_BYTES = TILE_XT + 12 * TILE_AT + TILE_DV + TILE_DVT;
constexpr int kJobs = 10;  // weight-gradient jobs: 4 layers x 2 row halves, W5 x 2

struct Bufs {
  int64_t tiles = 0;     // capacity in 128-row tiles
  int max_splits = 0;    // batch slices of the weight-gradient kernel
  uint8_t *img = nullptr;  // weight images (WIMG_BYTES)
  uint8_t *act = nullptr;  // tiles x TILE_BYTES
  uint8_t *xt = nullptr, *at[4] = {}, *dzt[4] = {}, *dv = nullptr, *dvt = nullptr;
  uint32_t *s[4] = {};
  float *ws = nullptr;   // max_splits x P_TOTAL
  // the rows of the following step, drawn by the weight-gradient kernel:
  // X0 [rows][32] and U [rows][4], valid for step pregen_step (-1: none)
  float *x0n = nullptr, *un = nullptr;
  int64_t pregen_step = -1;
};

// Buffers for batches of up to `batch` rows (images zeroed on `s`).
cudaError_t alloc(Bufs &b, int64_t batch, cudaStream_t s);
void release(Bufs &b);

struct Adam {
  float lr, b1, b2, eps, wd, bc1, bc2;
};

// Weight images from params (after begin, a loaded checkpoint).
cudaError_t pack(cudaStream_t s, Bufs &b, float *params);

// Forward, loss (added to *loss), backward and weight gradients of a batch of
// B rows, drawn in the forward kernel (gen non-null) or already in X0 [B][32]
// and U [B][4] (rows_early: written before the previous kernel ran, so the
// forward kernel may read them before its wait); the gradient lands in grad.
// With adam non-null the same launch that sums the gradient applies AdamW to
// params and repacks the weight images. With next non-null the
// weight-gradient kernel also draws the rows of step next->step into b.x0n /
// b.un (its epilogue warps, while the operands stream in).
cudaError_t step(cudaStream_t s, Bufs &b, int64_t B, const Gen *gen, const float *X0, const float *U,
                 bool rows_early, float *params, float *grad, float *m, float *v, const Adam *adam,
                 double *loss, int *err, const Gen *next = nullptr);

}  // namespace tf
}  // namespace gmc
