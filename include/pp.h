/*
 * pp.h -- C ABI of the urgency-served LiDAR pillar front end for NVIDIA GB300 (sm_103a).
 *
 * Two layers:
 *   1. Stage entry points (pp_voxelize, pp_pointnet, pp_scatter, pp_conv3x3, ...): one step of
 *      the pillar front end on device buffers the caller owns, enqueued on a caller stream.
 *   2. The serving runtime (pp_create ... pp_destroy, declared further below): chains, frame
 *      admission under an HBM budget, urgency-ordered batched release, completion polling.
 *
 * Conventions for every function here:
 *   - Return value is a pp_status: PP_OK (0) or a negative error.  Nothing aborts, throws or
 *     exits across this boundary.  A CUDA error seen while enqueueing returns PP_EDEVICE.
 *   - "device" pointers are CUDA device (or managed) addresses on the current device; "host"
 *     pointers are ordinary process memory.  No function takes ownership of a caller buffer.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Stage
 *     entry points only enqueue work; they never synchronise the stream.
 *   - Points are float4 (x, y, z, intensity) in metres, float32.  A batch of B frames is laid
 *     out as [B][cap_points][4] floats; frame b holds n_points[b] <= cap_points valid rows.
 *   - Activations are "padded NHWC": [B][H+2][W+2][C] with a one-pixel border that must be
 *     zero; ops write only the interior of their output unless stated otherwise.
 *
 * The method: the paper's 3D-perception chains (Section 6, Table 4: PointPillars, 22k-25k
 * points) are run here as a pillar front end -- voxelise, PointNet, BEV scatter, conv3x3
 * backbone -- and released by the urgency rules of Section 4 (Eq. 2, Sections 4.3-4.4.5).
 */
#ifndef PP_H_
#define PP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PP_OK = 0,
  PP_EINVAL = -1,     /* bad argument: null pointer, size out of range, unsupported shape   */
  PP_ENOMEM = -2,     /* device or host allocation failed                                    */
  PP_EAGAIN = -3,     /* not admitted now: HBM budget or frame slots exhausted; retry later  */
  PP_ETIMEDOUT = -4,  /* a bounded wait ran out                                              */
  PP_EDEVICE = -5,    /* a CUDA call failed, or a kernel reported a device-side error        */
  PP_ESTATE = -6      /* call not valid in the object's current state                        */
} pp_status;

/* Arithmetic types.  PP_F32 / PP_BF16 name a precision everywhere; PP_F32_TC is accepted only
 * by pp_scatter and the pp_conv_* calls and selects the FP32 conv on the tensor cores (3xTF32).
 * Its activations are "split FP32": two planes [2][B][H+2][W+2][C] of float, plane 0 the values
 * and plane 1 their TF32 remainders (x minus x with its 13 low mantissa bits cleared; see
 * pp_tf32_split), so that the conv reads both parts of its A operand by TMA. */
enum { PP_F32 = 0, PP_BF16 = 1, PP_F32_TC = 2 };

/* Pillar grid.  Ranges are half-open [min, max).  nx * vx must span x, ny * vy must span y.
 * max_pts must be 32.  Cell index of a point (binary32 arithmetic, round to nearest even, no
 * contraction): ix = floor((x - xmin) / vx), iy = floor((y - ymin) / vy); the point is kept iff
 * it lies inside all three ranges and 0 <= ix < nx, 0 <= iy < ny; cell = iy * nx + ix. */
typedef struct {
  float xmin, xmax, ymin, ymax, zmin, zmax, vx, vy;
  int32_t nx, ny, max_pillars, max_pts;
} pp_geometry;

/* Library version string, e.g. "pp 0.1 sm_103a". Never NULL. */
const char* pp_version(void);

/* Text of the last error recorded by this thread (empty string if none). Never NULL. */
const char* pp_last_error(void);

/* ---------------------------------------------------------------------------------------- */
/* Stage 1: voxelisation (point -> pillar).                                                  */
/*                                                                                           */
/* For each frame b: cell index per point (-1 = dropped); per-cell point counts via           */
/* warp-aggregated atomics; pillars = occupied cells in ascending cell order, at most         */
/* max_pillars of them; each pillar keeps the max_pts (32) points with the lowest input       */
/* indices, in ascending index order, gathered into pts (zero padded).  The result does not   */
/* depend on thread timing: it is bit-identical run to run.                                  */
/*                                                                                           */
/* Outputs (device, written for every frame; G = nx*ny, P = max_pillars):                    */
/*   cell           int32 [B][cap_points]   cell per point, -1 if dropped (rows >= n unset)   */
/*   cnt            uint32[B][G]            points per cell                                   */
/*   pillar_of_cell int32 [B][G]            pillar id of the cell, -1 if not a kept pillar    */
/*   coord          int32 [B][P]            cell of pillar p (p < num_pillars[b])             */
/*   npts           int32 [B][P]            min(count, 32) of pillar p                        */
/*   num_pillars    int32 [B]                                                                 */
/*   pts            float [B][P][32][4]     kept points of pillar p, zero rows after npts     */
/* Entries for p >= num_pillars[b] are unspecified.  n_points is a DEVICE array [B] so that a */
/* captured CUDA graph can be replayed with new counts; each value must be in [0, cap_points];*/
/* a value outside that range makes the frame empty and sets the error word in the workspace  */
/* (reported by pp_voxelize_check).                                                          */
/* workspace: device scratch of pp_voxelize_workspace_bytes() bytes, 256-byte aligned; its   */
/* first 256 bytes (the error word) must be zero before the first call; the rest needs no   */
/* initialisation.                                                                          */
size_t pp_voxelize_workspace_bytes(const pp_geometry* g, int32_t batch, int32_t cap_points);
int pp_voxelize(const pp_geometry* g, int32_t batch, int32_t cap_points,
                const float* points, const int32_t* n_points,
                int32_t* cell, uint32_t* cnt, int32_t* pillar_of_cell,
                int32_t* coord, int32_t* npts, int32_t* num_pillars, float* pts,
                void* workspace, size_t workspace_bytes, void* stream);
/* Synchronises `stream`, then reads the workspace's error word: PP_OK or PP_EINVAL (a
 * n_points value was out of range). */
int pp_voxelize_check(const void* workspace, void* stream);

/* pp_voxelize followed by pp_pointnet as a release unit runs them: the point selection is fused
 * into the PointNet kernel (each warp picks its pillar's 32 lowest point indices and loads the
 * points straight into registers), so there is no pts output and the gathered points never go
 * through memory.  Arguments as for the two calls (pfn_w, scale_shift, feat as pp_pointnet's);
 * every output, feat included, is bit-identical to pp_voxelize + pp_pointnet on the same input.
 * Workspace: pp_voxelize_workspace_bytes(); pp_voxelize_check reads its error word. */
int pp_voxelize_pointnet(const pp_geometry* g, int32_t batch, int32_t cap_points, const float* points,
                         const int32_t* n_points, int32_t* cell, uint32_t* cnt, int32_t* pillar_of_cell,
                         int32_t* coord, int32_t* npts, int32_t* num_pillars, const float* pfn_w,
                         const float* scale_shift, float* feat, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Same operation and outputs as pp_voxelize, for callers that cannot allocate device memory:
 * the paper has no counterpart; this entry point exists for deployments such as real-time
 * task threads that may not call the CUDA allocator once they run (cudaMalloc/cudaFree can
 * block or synchronise the whole device) and hosts whose device memory is owned by another
 * framework.  It takes no workspace: its scratch is a file-scope device array of
 * PP_VOX_STATIC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library holds until
 * the process exits.  Calls needing more scratch than that (pp_voxelize_workspace_bytes() >
 * PP_VOX_STATIC_SCRATCH_BYTES, e.g. batch 8 x 150,000 points fits, 16 x 150,000 does not)
 * return PP_EINVAL with a message and enqueue nothing.  It allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and caches it; make
 * that first call before any stream capture.  All calls share the one array, which keeps the
 * previous call's contents (the call clears the part that must start at zero): calls whose
 * work overlaps on the GPU (concurrent streams, or threads) race on it and must be
 * serialised by the caller.  A n_points value outside [0, cap_points] makes that frame empty
 * (this variant has no error word to report it). */
#define PP_VOX_STATIC_SCRATCH_BYTES (16u << 20)
int pp_voxelize_static(const pp_geometry* g, int32_t batch, int32_t cap_points,
                       const float* points, const int32_t* n_points,
                       int32_t* cell, uint32_t* cnt, int32_t* pillar_of_cell,
                       int32_t* coord, int32_t* npts, int32_t* num_pillars, float* pts,
                       void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Stage 2: PointNet.  Per pillar p < num_pillars[b] and channel c < 64:                     */
/*   features f = (x, y, z, r, x-mx, y-my, z-mz, x-xc, y-yc) per kept point, where (mx,my,mz)*/
/*   is the mean of the pillar's kept points and (xc, yc) = (xmin + (ix+.5) vx,              */
/*   ymin + (iy+.5) vy) is its cell centre;                                                  */
/*   feat[b][p][c] = max over the kept points of ReLU(scale[c] * (W[c] . f) + shift[c]).     */
/* pfn_w: device float [64][9] (Linear weight, no bias).  scale_shift: device float [2][64]  */
/* (inference BN folded, see pp_bn_fold).  feat: device float [B][P][64]; rows p >=           */
/* num_pillars[b] are unspecified.  Computed in FP32.                                        */
int pp_pointnet(const pp_geometry* g, int32_t batch, const float* pts, const int32_t* npts,
                const int32_t* coord, const int32_t* num_pillars, const float* pfn_w,
                const float* scale_shift, float* feat, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Stage 3: BEV scatter.  Writes the WHOLE padded canvas [B][ny+2][nx+2][64] (dtype PP_F32   */
/* or PP_BF16, round to nearest even): interior pixel (iy, ix) gets feat[b][p] if            */
/* pillar_of_cell[b][iy*nx+ix] = p >= 0, else zeros; the border is zero.  One coalesced pass, */
/* so no separate clear is needed.  PP_F32_TC writes the split FP32 canvas: the PP_F32 canvas */
/* as plane 0 and its TF32 remainders as plane 1 ([2][B][ny+2][nx+2][64]).                   */
int pp_scatter(const pp_geometry* g, int32_t batch, const float* feat,
               const int32_t* pillar_of_cell, void* canvas, int32_t dtype, void* stream);

/* Stage 3, incremental: the same canvas as pp_scatter for a canvas that persists from frame to
 * frame (a release unit's), writing only what changes: the cells drawn for the previous frame
 * that hold no kept pillar now are zeroed, then every kept pillar p < num_pillars[b] is written
 * at coord[b][p] (values, TF32 remainders for PP_F32_TC, or BF16 round to nearest even), and
 * drawn[b][0..num_pillars[b]) / drawn_num[b] are set to this frame's cells.  Traffic is about
 * 2 x pillars x 64 x element size instead of the whole canvas.  State (device memory the caller
 * owns): canvas, drawn int32 [B][P] and drawn_num int32 [B]; start from a zero canvas (border
 * included) and drawn_num = 0, and pass the same three with every frame of that batch row.
 * Afterwards the canvas equals pp_scatter's for this frame, bit for bit.  coord, num_pillars,
 * pillar_of_cell: pp_voxelize's outputs for the frame. */
int pp_scatter_update(const pp_geometry* g, int32_t batch, const float* feat, const int32_t* coord,
                      const int32_t* num_pillars, const int32_t* pillar_of_cell, int32_t* drawn,
                      int32_t* drawn_num, void* canvas, int32_t dtype, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Stage 4: one backbone layer, conv3x3 (zero pad 1, stride 1 or 2, no bias) + folded BN +    */
/* ReLU, implicit GEMM over padded NHWC.                                                     */
/*   in : [B][H+2][W+2][cin]  of dtype, border zero (PP_F32_TC: [2][B][H+2][W+2][cin] split  */
/*        FP32, see PP_F32_TC)                                                               */
/*   out: [B][Ho+2][Wo+2][cout] of dtype, Ho = (H-1)/stride + 1, Wo = (W-1)/stride + 1; only  */
/*        the interior is written (the border must already be zero).  PP_F32_TC: both planes */
/*        [2][B][Ho+2][Wo+2][cout] are written, plane 1 = TF32 remainders of plane 0.         */
/*   w  : packed weights from pp_conv_pack_weights for the same dtype.                       */
/*   scale_shift: device float [2][cout].                                                    */
/* PP_F32: CUDA-core FP32 FMA.  PP_BF16: tcgen05 tensor cores, BF16 x BF16 -> FP32 in TMEM,   */
/* BF16 output.  PP_F32_TC: FP32 in and out on the tcgen05 tensor cores: each operand split   */
/* into a TF32 part and an FP32 remainder, three kind::tf32 products accumulated in FP32     */
/* (error of the order of FP32 rounding).  cin, cout multiples of 64; stride 2 needs even H, W.*/
/* tile: -1 = library choice (autotuned table when present), else an index into the tile     */
/* list of pp_conv_tile_count(dtype).                                                        */
int pp_conv3x3(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t stride,
               int32_t dtype, const void* in, const void* w, const float* scale_shift,
               void* out, int32_t tile, void* stream);
/* pp_conv3x3 with a workspace for the stream-K tiles of PP_F32_TC (the K blocks of all output
 * tiles laid end to end and cut into one equal range per SM; a tile split between SMs is
 * finished by the last of them, from partial sums in the workspace).  workspace: device, 256-
 * byte aligned, >= pp_conv_workspace_bytes() bytes, zero-filled before its first use; every
 * completed launch leaves it ready for the next (a launch that failed on the device leaves it
 * unspecified: zero it again).  Launches that share a workspace must be stream-ordered.  With
 * workspace NULL, stream-K tiles return PP_EINVAL, and tile = -1 falls back to the same tile
 * without stream-K.  Results of a stream-K tile differ from the plain tile's only by FP32
 * rounding (the partial sums are added in a fixed order, so a given shape, batch and tile is
 * bit-reproducible). */
int pp_conv3x3_ws(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t stride,
                  int32_t dtype, const void* in, const void* w, const float* scale_shift,
                  void* out, int32_t tile, void* workspace, size_t workspace_bytes, void* stream);
/* Workspace bytes pp_conv3x3_ws needs for every stream-K tile of this shape (0: none). */
size_t pp_conv_workspace_bytes(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                               int32_t stride, int32_t dtype);
int pp_conv_tile_count(int32_t dtype);
/* Shape of conv tile `tile` of `dtype`: output box bh x bw pixels (bh*bw = 128 on the tensor
 * cores; CUDA-core tiles report bh = 1, bw = pixels per tile), bn output channels, and whether
 * the kernel is persistent: 1 = one CTA per SM walking the tiles, TMA ring and TMEM
 * accumulators carried across tiles (the default for the tensor-core dtypes); 2 = the BF16
 * row-streaming kernel for 64 -> 64 channel layers (the default there: weights resident in
 * shared memory, each input row loaded once and every tap read as a row-shifted view; tile
 * reports the 128-pixel output row segment; the last two BF16 tiles, strips of output rows cut
 * for about two strips per SM, or one longer strip each); 3 = persistent with the stream-K
 * partition (PP_F32_TC; needs a workspace, see pp_conv3x3_ws); 4 = persistent over runs of
 * 128 consecutive output pixels (the output laid out over the padded width) whose three kx taps
 * share one loaded 130-pixel input range (PP_F32_TC, the six tiles before the last: 64 and 128 output
 * channels, then the same with deeper rings; stride 1 and cout a multiple of bn only, PP_EINVAL
 * otherwise); 5 = the first two of those with the stream-K partition (the accumulation groups of
 * one ky and one 32-channel chunk of all tiles cut into one equal range per SM; needs a
 * workspace like 3); 6 = persistent over runs of 126 consecutive output pixels (bw = 126) with
 * the three kx taps' 64 output channels side by side in the MMA's N dimension and the kx shift
 * applied to the accumulator rows (PP_F32_TC, the last tile; stride 1 and cout a multiple of
 * 64 only, PP_EINVAL otherwise). */
int pp_conv_tile_info(int32_t dtype, int32_t tile, int32_t* bh, int32_t* bw, int32_t* bn,
                      int32_t* persistent);

/* Conv tile autotuner (this library's; the tile choice of the layers is not from the paper).
 * Runs every tile of `dtype` that supports the shape on the given buffers (same meaning as
 * pp_conv3x3; `out` holds a valid result afterwards), timing `reps` launches of each by one
 * replay of a captured CUDA graph, and records the fastest for this (dtype, shape): from then
 * on tile = -1 in pp_conv3x3 and in release units means that tile.  Synchronous (uses and
 * destroys a private stream).  *best_us (may be NULL) = device time per launch. */
int pp_conv_autotune(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                     int32_t stride, int32_t dtype, const void* in, const void* w,
                     const float* scale_shift, void* out, int32_t reps, int32_t* best_tile,
                     float* best_us);
/* pp_conv_autotune that also times the stream-K tiles, on `workspace` (see pp_conv3x3_ws). */
int pp_conv_autotune_ws(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout,
                        int32_t stride, int32_t dtype, const void* in, const void* w,
                        const float* scale_shift, void* out, void* workspace,
                        size_t workspace_bytes, int32_t reps, int32_t* best_tile, float* best_us);
/* Writes the autotuned table as text ("dtype batch H W cin cout stride tile us" per line). */
int pp_conv_tune_save(const char* path);
/* Reads a table written by pp_conv_tune_save (host only, no GPU needed); returns the number of
 * entries loaded (>= 0) or a negative pp_status.  Lines naming a tile that does not exist are
 * skipped. */
int pp_conv_tune_load(const char* path);
/* Forgets every autotuned entry. */
void pp_conv_tune_clear(void);

/* ---------------------------------------------------------------------------------------- */
/* Neck and detection head (the rest of PointPillars' GPU segment; the paper runs it inside a */
/* closed engine and does not describe it): each backbone block's output is upsampled to the  */
/* first block's size by a transposed conv whose kernel equals its stride (no overlap) + BN + */
/* ReLU, the upsampled maps are concatenated along channels, and a 1x1 conv with bias gives   */
/* the per-anchor outputs.  Both run on the persistent tensor-core GEMM (dtype PP_BF16, or    */
/* PP_F32_TC with split FP32 operands and outputs).                                            */
/* pp_upsample: in [B][H+2][W+2][cin] -> channels [out_coff, out_coff + cout) of out          */
/*   [B][up*H+2][up*W+2][out_c] (interior written: out[up*y+dy][up*x+dx][out_coff+co] =        */
/*   ReLU(scale[co] * sum_ci in[y][x][ci] w[ci][co][dy][dx] + shift[co])).  cin, cout, out_c,   */
/*   out_coff multiples of 64; scale_shift device [2][cout] (pp_bn_fold).                       */
/* pp_head: out[B][H+2][W+2][cout_pad] = in . w^T + bias (no activation), cout_pad = cout     */
/*   rounded up to a multiple of 64 (the extra channels are 0); scale_shift device [2][cout_pad] */
/*   from pp_head_pack_weights (1 and the bias).                                                */
/* The *_packed_bytes calls return 0 for a shape or dtype the GEMM does not support.           */
/* Weights are packed on the host and copied to device memory (synchronous): pp_upsample_*    */
/* from the ConvTranspose2d layout [cin][cout][up][up], pp_head_* from [cout][cin].  tile: a  */
/* tile number whose pp_conv_tile_info persistent flag is 1 (its bn must divide cout), or -1  */
/* for the library's choice.  Returns PP_EINVAL (nothing launched) for a bad shape, alignment */
/* or tile; all pointers are device memory owned by the caller, except the host weights.     */
size_t pp_upsample_packed_bytes(int32_t cin, int32_t cout, int32_t up, int32_t dtype);
int pp_upsample_pack_weights(const float* w, int32_t cin, int32_t cout, int32_t up, int32_t dtype,
                             void* w_packed);
size_t pp_head_packed_bytes(int32_t cin, int32_t cout, int32_t dtype);
int pp_head_pack_weights(const float* w, const float* bias, int32_t cin, int32_t cout, int32_t dtype,
                         void* w_packed, float* scale_shift);
int pp_upsample(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t up, int32_t dtype,
                const void* in, const void* w_packed, const float* scale_shift, void* out, int32_t out_c,
                int32_t out_coff, int32_t tile, void* stream);
int pp_head(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dtype, const void* in,
            const void* w_packed, const float* scale_shift, void* out, int32_t tile, void* stream);

/* TF32 remainder plane of n floats (device): lo[i] = x[i] - (x[i] with its 13 low mantissa
 * bits cleared), exact in FP32 (the part a TF32 read of x[i] drops).  Turns an FP32 tensor into
 * the split FP32 form of PP_F32_TC (x as plane 0, lo as plane 1).  x and lo may not overlap. */
int pp_tf32_split(const float* x, float* lo, int64_t n, void* stream);

/* Repacks float OIHW weights [cout][cin][3][3] (device) into the layout pp_conv3x3 expects
 * for `dtype` (device, pp_conv_packed_bytes() bytes): PP_F32 -> [9*cin][cout] float,
 * PP_BF16 -> [cout][9*cin] bf16 (round to nearest even), PP_F32_TC -> [2][cout][9*cin] float
 * (plane 0: weight with the 13 low mantissa bits cleared, plane 1: the remainder);
 * K index = (ky*3+kx)*cin + ci.  cin and cout multiples of 64, as pp_conv3x3 takes them (else
 * 0 bytes / PP_EINVAL: pp_conv3x3 reads 9*cin*cout weights from the buffer it is given). */
size_t pp_conv_packed_bytes(int32_t cin, int32_t cout, int32_t dtype);
int pp_conv_pack_weights(const float* w_oihw, int32_t cin, int32_t cout, int32_t dtype,
                         void* w_packed, void* stream);

/* Host helper: folds inference BN rows (gamma, beta, mean, var) [4][c] (host float) into
 * scale = gamma / sqrt(var + eps), shift = beta - mean * scale, written to out [2][c] (host
 * float), computed in double.  eps is the BN epsilon (1e-3 for this network). */
int pp_bn_fold(const float* bn, int32_t c, float eps, float* out);

/* Reads the library's sticky device error word (bit 1: a TMA producer wait timed out, bit 2: an
 * MMA wait timed out, bit 4: an epilogue wait timed out in the tensor-core conv; the kernel
 * that hit it skipped its stores).  Synchronous (device-wide copy).  clear != 0 resets it. */
int pp_device_error(uint32_t* code, int32_t clear);
/* Sets `bits` in that word, as a bounded wait that ran out would (no counterpart in the paper:
 * a hook for testing the error path without a device fault).  Every tensor-core conv launched
 * while it is set exits at once without writing its outputs, and a release unit that finds it
 * set reports its frames as PP_FRAME_ERROR.  Synchronous; pp_device_error(.., 1) clears it. */
int pp_device_error_set(uint32_t bits);

/* ======================================================================================== */
/* Serving runtime.                                                                          */
/*                                                                                           */
/* Chains release frames periodically (Section 4.1); each frame runs the pillar front end and */
/* must finish by its absolute deadline.  The runtime admits frames under a fixed HBM budget, */
/* keeps admitted frames on the host until release, and a dispatcher thread releases them in  */
/* units of up to max_batch frames (one CUDA-graph launch per unit) following the paper's     */
/* rules: urgency UL = 1/slack (Eq. 2), early exit of frames whose slack is negative          */
/* (Section 4.3), task-level stream binding with a reserved top priority (Section 4.4.3),     */
/* delayed launching behind urgent units of other chains (Section 4.4.4), and batched launch  */
/* synchronisation with overlap (Section 4.4.5).  Policy PP_POLICY_FIFO is the plain baseline:*/
/* every frame launched on arrival on its chain's default-priority stream, kernel by kernel,  */
/* no graph, no batching, no urgency.  The other policies are the textbook orders the paper */
/* compares against (Section 6.4, comparison of policies; not defined there): they replace the */
/* urgency order and its stream ranking, with no early exit, reservation or delaying:         */
/*   PP_POLICY_EDF   earliest absolute deadline first;                                        */
/*   PP_POLICY_SJF   shortest remaining estimate (est_gpu + est_cpu) first;                   */
/*   PP_POLICY_HRRN  highest response ratio (waiting + estimate) / estimate first;            */
/*   PP_POLICY_LCUF  lowest chain utilisation (estimate / period) first;                      */
/*   PP_POLICY_SAEDF slack-aware EDF: frames that can still meet their deadline (slack >= 0)  */
/*                   by earliest deadline, then the others by earliest deadline;             */
/*   PP_POLICY_EQDF  earliest quasi-deadline (deadline - eqdf_lambda x estimate) first.       */
/* Times are microseconds on the host monotonic clock (pp_now_us).                           */
/* Threading: every entry point may be called from any thread; one internal dispatcher       */
/* thread does the rest.                                                                     */

enum { PP_POLICY_FIFO = 0, PP_POLICY_URGENCY = 1, PP_POLICY_EDF = 2, PP_POLICY_SJF = 3,
       PP_POLICY_HRRN = 4, PP_POLICY_LCUF = 5, PP_POLICY_SAEDF = 6, PP_POLICY_EQDF = 7 };
enum { PP_FRAME_DONE = 0, PP_FRAME_DROPPED = 1, PP_FRAME_ERROR = 2 };
#define PP_MAX_BLOCKS 4
#define PP_MAX_CHAINS 64

typedef struct {
  pp_geometry geom;
  /* backbone: block b has convs[b] conv3x3 layers of chans[b] channels, the first one with
   * stride strides[b] (the others stride 1).  Input channels of the first layer: 64. */
  int32_t n_blocks, convs[PP_MAX_BLOCKS], chans[PP_MAX_BLOCKS], strides[PP_MAX_BLOCKS];
  /* weights, host float, copied by pp_create: pfn_w [64][9]; pfn_bn [4][64]; per layer
   * conv_w[l] [cout][cin][3][3] and conv_bn[l] [4][cout].  BN rows: gamma, beta, mean, var;
   * epsilon 1e-3. */
  const float* pfn_w;
  const float* pfn_bn;
  const float* const* conv_w;
  const float* const* conv_bn;
  int32_t max_batch;            /* frames per release unit, 1..8                              */
  int32_t cap_points;           /* maximum points per frame                                   */
  int32_t precisions;           /* bit 0: FP32 units, bit 1: BF16 units                       */
  int32_t units;                /* units per precision; 0 = as many as the budget allows (16) */
  uint64_t hbm_budget_bytes;    /* device memory the context may hold (units + staging)       */
  int32_t policy;               /* PP_POLICY_* (FIFO, URGENCY, EDF, SJF, HRRN, LCUF)          */
  int32_t use_graphs;           /* replay one CUDA graph per unit launch                      */
  double delta_eval_us;         /* batch closes when its estimated GPU time reaches this      */
  int32_t max_closed;           /* closed batches allowed in flight: 2 overlapped, 1 sync,    */
                                /* 0 = no synchronisation                                     */
  double delay_quantum_us;      /* re-check period of a delayed release                       */
  double th_urgent;             /* UL threshold (1/us); 0 = calibrate, < 0 = off              */
  int32_t th_calib_frames;      /* frames sampled for the calibration (p95 of max UL)         */
  double util_exempt;           /* units below this utilisation are never delayed             */
  int32_t early_exit;           /* drop frames whose slack is negative                        */
  int32_t num_streams;          /* stream priority levels per chain; 0 = device range         */
  int32_t max_admitted;         /* admitted-but-unreleased frames per precision (each holds a  */
                                /* result slot in HBM); 0 = as many as the budget allows, the  */
                                /* library caps it at 128                                      */
  int32_t fp32_cuda_cores;      /* FP32 convs on CUDA cores (1) or on the tensor cores with the */
                                /* 3xTF32 split (0, default)                                   */
  int32_t autotune;             /* autotune every conv layer for each unit size at creation     */
                                /* (pp_conv_autotune; default 1)                               */
  int32_t stream_k;             /* let the autotuner pick stream-K tiles for 3xTF32 convs (each */
                                /* unit then owns a workspace).  Within FP32 tolerance either  */
                                /* way, but a frame's result is bit-identical across unit sizes */
                                /* only without it (default 0)                                 */
  /* Neck and detection head (head_outputs = 0: a unit ends at the backbone).  Block b's output
   * is upsampled to block 0's size by a transposed conv of kernel = stride = s_b (block 0's
   * height / block b's height, equal for the width) + BN + ReLU into up_channels channels at
   * channel offset b * up_channels of the neck map, and the 1x1 head with bias maps that to
   * head_outputs channels (pp_upsample / pp_head).  Tensor-core convs only (fp32_cuda_cores =
   * 0).  Weights host float, copied by pp_create: up_w[b] [chans[b]][up_channels][s_b][s_b],
   * up_bn[b] [4][up_channels], head_w [head_outputs][n_blocks * up_channels], head_b
   * [head_outputs]. */
  int32_t head_outputs;         /* 1..1024, or 0                                               */
  int32_t up_channels;          /* multiple of 64 (default 128)                                */
  const float* const* up_w;
  const float* const* up_bn;
  const float* head_w;
  const float* head_b;
  double eqdf_lambda;           /* PP_POLICY_EQDF's estimate weight (default 0.5)              */
  /* Estimate-noise experiment (the paper's study of urgency estimation error): every frame's   */
  /* GPU-time estimate, as the release policy sees it, is scaled by pp_noise_factor(noise_seed, */
  /* frame id, est_noise), drawn once per frame.  0 = off (default).                           */
  double est_noise;             /* half-width eps of the uniform factor 1 + U[-eps, eps), < 1 */
  uint64_t noise_seed;
  int32_t keep_blocks;          /* result slots hold every backbone block's output (1) or only */
                                /* the last block's, the final output (0, default)            */
  int32_t decision_log;         /* record the first decision_log release decisions with their */
                                /* inputs (pp_decision_log); 0 = off (default), at most 2^20   */
} pp_config;

/* Fills *cfg with defaults for the given geometry/backbone-free fields (policy urgency,
 * max_batch 8, delta_eval 500 us, max_closed 2, delay quantum 1000 us, th_urgent 0 (calibrate
 * over 64 frames), util_exempt 0.1, early_exit 1, graphs on, both precisions, budget 20 GiB).
 * The paper's values: Delta_eval 0.5 ms and overlapped batches (Section 4.4.5), a 1 ms sleep
 * loop and the 0.1 utilisation exemption (Section 4.4.4), TH_urgent at the 95th percentile of
 * the highest urgency sampled (Section 4.4.3). */
void pp_config_defaults(pp_config* cfg);

typedef struct pp_ctx pp_ctx;

/* Creates a context on the current CUDA device: uploads weights, allocates the units (each
 * holding buffers for max_batch frames), captures their graphs, carves one result slot per
 * admissible frame out of what is left of the budget, and starts the dispatcher.  A unit is
 * reusable as soon as it completes: it copies its frames' block outputs into their result
 * slots.  PP_ENOMEM if one unit per enabled precision and one result slot do not fit.
 * Paper: the offline profiling stage and its lookup table of execution times (Section 4.1,
 * Table 1) -- here every unit size is timed once at creation to seed the per-(precision,
 * frames-per-unit) estimates, each later the mean of its last 8 measured launches (the moving
 * average of Section 4.2).  The HBM admission budget has no counterpart in the paper.
 * Ownership: the context owns every device buffer it allocates until pp_destroy; weights are
 * copied.  Errors: PP_EINVAL for a bad config, PP_ENOMEM, PP_EDEVICE. */
int pp_create(const pp_config* cfg, pp_ctx** out);

/* Declares a chain.  period/deadline in milliseconds (informational/default deadline);
 * precision PP_F32 or PP_BF16 (needs that precision enabled).  Up to PP_MAX_CHAINS ids,
 * 0 <= chain_id < PP_MAX_CHAINS.  Paper: the task chain with its application-defined deadline
 * and its period (Section 4.1; Table 2 lists chains by period, deadline and estimates).  The
 * chain gets its own pool of streams, one per device stream priority (the per-task stream pool
 * of Section 4.4.3).  Errors: PP_EINVAL (bad id, period, deadline or precision), PP_ESTATE
 * (already registered), PP_EDEVICE (stream creation). */
int pp_register_chain(pp_ctx* ctx, int32_t chain_id, double period_ms, double rel_deadline_ms,
                      int32_t precision);

/* Declares a synthetic-load chain (the paper's robustness study with custom kernels of set
 * utilisation and execution time, Section 6.6): each of its frames runs n_kernels launches of
 * a vector-add style kernel on round(util x SMs) CTAs (each holds an SM alone, so util is the
 * fraction of the GPU it occupies), each launch calibrated once here to last about kernel_us.  Its frames
 * are submitted like any other (points ignored, n_points 0), released by the same policy
 * (utilisation util for the delay exemption; estimates from the chain's own measured
 * durations, n_kernels x kernel_us before the first), run one per unit, and complete with no
 * outputs (out_dev NULL, out_dtype -1).  n_kernels 1..256, kernel_us 1..100000, util (0, 1],
 * at most 1 s of kernels per frame.  Synchronous (a few ms of calibration launches). */
int pp_register_synthetic_chain(pp_ctx* ctx, int32_t chain_id, double period_ms, double rel_deadline_ms,
                                int32_t n_kernels, double kernel_us, double util);

/* Where submitted points live (the is_device_ptr argument):
 *   PP_POINTS_HOST (0)   host memory, copied into a pinned staging slot before the call returns;
 *   PP_POINTS_DEVICE (1) device memory, borrowed until the frame's result is polled;
 *   PP_POINTS_PINNED (2) page-locked host memory (cudaHostAlloc / cudaHostRegister, e.g. a
 *                        pinned torch tensor), borrowed until the frame's result is polled;
 *                        no staging copy: a release unit of one frame reads it in place over
 *                        the host link from its own kernels; a unit batching several frames
 *                        copies it by copy engine into the unit's device point slot ahead of
 *                        its kernels (in the unit's stream).  Other host memory: PP_EINVAL. */
enum { PP_POINTS_HOST = 0, PP_POINTS_DEVICE = 1, PP_POINTS_PINNED = 2 };
/* Submits one frame of `n_points` float4 points (is_device_ptr: PP_POINTS_*; device and pinned
 * points 16-byte aligned).
 * t_arrival_us / abs_deadline_us on the pp_now_us clock (abs_deadline_us <= 0: arrival +
 * the chain's deadline).  PP_EAGAIN when admitting the frame would exceed the HBM budget.
 * Paper: a frame's arrival starts an instance of its chain, with t_arr and D as in Eq. 2
 * (Section 4.2); its urgency is evaluated from then on at every release decision.  The frame
 * (its staged points and its result slot) is the unit of admission here, which the paper does
 * not have.  Layout: float4 (x, y, z, intensity) per point. */
int pp_submit_frame(pp_ctx* ctx, int32_t chain_id, const float* xyzr, int64_t n_points,
                    int32_t is_device_ptr, double t_arrival_us, double abs_deadline_us,
                    uint64_t* frame_id_out);

/* Submits n (1..PP_MAX_SUBMIT) frames at once, all arriving at t_arrival_us: they become ready
 * together, so that one release decision can batch them into a single unit (uneven point
 * counts share the unit's graph).  chain_ids / xyzr / n_points: host arrays of n entries, same
 * meaning as in pp_submit_frame; abs_deadline_us: n deadlines, or NULL for each chain's own.
 * Frames are admitted in order until one cannot be: *n_admitted (may be NULL) receives how
 * many were, frame_ids_out (may be NULL) their ids, and the call returns PP_EAGAIN (budget
 * full) or PP_ENOMEM for the first frame left out.  Argument errors admit no frame.
 * Paper: arrivals as in pp_submit_frame (Section 4.2); admitting them under one lock makes
 * them one ready set at the next decision, which may release them as one unit -- the batching
 * of several chains' frames into one launch has no counterpart in the paper (its kernels are
 * per task). */
#define PP_MAX_SUBMIT 64
int pp_submit_frames(pp_ctx* ctx, int32_t n, const int32_t* chain_ids, const float* const* xyzr,
                     const int64_t* n_points, int32_t is_device_ptr, double t_arrival_us,
                     const double* abs_deadline_us, uint64_t* frame_ids_out, int32_t* n_admitted);
/* pp_submit_frames with a host output buffer per frame: host_out[i] (host array of n pointers,
 * may be NULL, entries may be NULL) is page-locked host memory of pp_result_bytes() bytes for
 * the frame's precision, 16-byte aligned, borrowed until the frame is polled.  The unit writes
 * the frame's final output (the out_dev map: last backbone block, or the head) there as part of
 * the same launch (a one-frame unit from its result copy kernel over the host link; a unit
 * batching several frames by one copy-engine copy per frame after its kernels, in its stream),
 * so a caller that wants its result on the host needs no copy of its own (pp_result.out_host;
 * complete when the frame is polled).  Other host memory: PP_EINVAL,
 * nothing admitted.  Ignored for synthetic-load chains.  Paper: as pp_submit_frames; the
 * output buffer (results delivered to host memory by the unit) has no counterpart in the
 * paper. */
int pp_submit_frames_ex(pp_ctx* ctx, int32_t n, const int32_t* chain_ids, const float* const* xyzr,
                        const int64_t* n_points, int32_t is_device_ptr, double t_arrival_us,
                        const double* abs_deadline_us, void* const* host_out, uint64_t* frame_ids_out,
                        int32_t* n_admitted);
/* Bytes of one frame's final output (padded NHWC, out_dev's map) at `precision` (0 if that
 * precision is not enabled).  No counterpart in the paper (a size query for host buffers). */
size_t pp_result_bytes(pp_ctx* ctx, int32_t precision);

typedef struct {
  uint64_t frame_id;
  int32_t chain_id;
  int32_t status;               /* PP_FRAME_DONE / PP_FRAME_DROPPED / PP_FRAME_ERROR          */
  double t_arr_us, t_release_us, t_done_us, deadline_us;
  int32_t missed;               /* t_done > deadline, or dropped                              */
  int32_t num_pillars;
  int32_t batch;                /* frames in the unit this frame ran in                       */
  int32_t level;                /* stream priority level it was released on (0 = highest)     */
  const void* out_dev;          /* last backbone layer (or the head), padded NHWC            */
                                /* [out_h+2][out_w+2][out_c]                                  */
  int32_t out_c, out_h, out_w, out_dtype;
  const void* block_dev[PP_MAX_BLOCKS];  /* output of each block kept (keep_blocks: all; else  */
                                         /* the last block's only, others NULL), same layout   */
  int32_t block_c[PP_MAX_BLOCKS], block_h[PP_MAX_BLOCKS], block_w[PP_MAX_BLOCKS];
  /* with a head (head_outputs > 0): out_dev is the head map [out_h+2][out_w+2][out_c] at block */
  /* 0's size, out_c = head_outputs rounded up to 64 (channels past out_valid_c are 0), and the */
  /* block outputs are not kept (block_dev NULL); without one out_valid_c = out_c.              */
  int32_t out_valid_c;
  /* frames submitted with a host output buffer (pp_submit_frames_ex): that buffer, holding a  */
  /* copy of out_dev ([out_h+2][out_w+2][out_c]), complete when the frame is polled; else NULL */
  const void* out_host;
} pp_result;

/* Drains up to `max` completed frames into out[]; waits up to timeout_us for the first one
 * (0 = do not wait).  *n_out = number written (0 on timeout, return PP_OK).  Output buffers
 * (the frame's result slot) stay valid until pp_result_release(frame_id), which returns the
 * slot to the budget.  A frame dropped by early exit carries no outputs (out_dev NULL) and
 * gives its slot back at once; releasing it only forgets the record.  A frame whose unit
 * failed on the device comes back with status PP_FRAME_ERROR (the call still returns PP_OK;
 * pp_stats counts such units).  Paper: completion is where an active kernel's record leaves
 * the Active Kernel Buffer (Section 4.4.2) and a batch's synchronisation point is passed
 * (Section 4.4.5); latency and misses follow the metrics of Section 6.2. */
int pp_poll(pp_ctx* ctx, pp_result* out, int32_t max, int32_t* n_out, int64_t timeout_us);
/* Returns a polled frame's result slot to the HBM budget (no counterpart in the paper: its
 * outputs are the application's).  PP_EINVAL for an unknown id, PP_ESTATE if not completed. */
int pp_result_release(pp_ctx* ctx, uint64_t frame_id);
/* pp_result_release for n frames under one lock; every id is tried, and the first error met
 * (unknown or not completed) is returned.  No counterpart in the paper, as pp_result_release. */
int pp_result_release_many(pp_ctx* ctx, int32_t n, const uint64_t* frame_ids);

typedef struct {
  uint64_t submitted, done, dropped, missed, rejected;
  double overall_miss_ratio;     /* Eq. 3: mean over chains of misses / frames               */
  double lat_p50_us, lat_p99_us, lat_mean_us;
  double frames_per_s;           /* completed frames / (last done - first arrival)           */
  uint64_t units_launched;
  double mean_batch;
  uint64_t delayed_releases;
  double delayed_us;
  uint64_t collisions;           /* launches made while another chain's urgent unit ran      */
  double sched_us_per_decision;
  double th_urgent;              /* threshold in use (1/us)                                  */
  uint64_t chain_frames[PP_MAX_CHAINS], chain_missed[PP_MAX_CHAINS];
  double chain_p99_us[PP_MAX_CHAINS];
  uint64_t device_errors;        /* units whose launch failed, whose completion event reported */
                                 /* an error, or whose kernels found a device error word set;  */
                                 /* their frames completed with PP_FRAME_ERROR                 */
  uint32_t device_error_code;    /* the last nonzero device error word a unit reported (bits   */
                                 /* of pp_device_error; bit 31: voxeliser point count)         */
  uint64_t decisions;            /* calls of the release rule made by the dispatcher          */
} pp_stats;

/* Counters and latency percentiles so far.  overall_miss_ratio is Eq. 3 (Section 6.2): the mean
 * over chains of each chain's missed / total instances (a dropped or failed frame is a miss);
 * collisions as counted for Section 4.4.3.  `out` is a caller struct of sizeof(pp_stats)
 * (pp_struct_size("pp_stats") gives this build's size). */
int pp_get_stats(pp_ctx* ctx, pp_stats* out);
/* Starts the statistics afresh (counters, latency samples, per-chain counts, the decision count;
 * the estimate table, TH_urgent and every frame in flight are kept): a measurement that excludes
 * a warm-up phase.  The paper evaluates after its chains have run in (Section 6.1); no
 * counterpart as an entry point. */
int pp_stats_reset(pp_ctx* ctx);
/* Stops the dispatcher, waits (bounded, 10 s) for in-flight units, frees everything.
 * PP_ETIMEDOUT if the device did not finish in time (resources are then leaked, not freed).
 * No counterpart in the paper (its chains run for the life of the process). */
int pp_destroy(pp_ctx* ctx);
/* Host monotonic clock in microseconds: the clock of t_arr, D and t in Eq. 2 (the paper reads
 * clock_gettime, Section 4.2). */
double pp_now_us(void);
/* sizeof of a public struct, by its type name ("pp_config", "pp_result", "pp_stats",
 * "pp_geometry", "pp_arrival", "pp_replay_stats", "pp_policy_frame", "pp_policy_active",
 * "pp_policy_config", "pp_policy_decision", "pp_decision_record"); 0 for any other name.  Lets a binding check its
 * struct mirrors against this build.  No counterpart in the paper (ABI versioning). */
size_t pp_struct_size(const char* type_name);
/* The estimate-noise factor of frame `frame_id`: 1 + eps (2u - 1) with u = the frame_id-th
 * output of a SplitMix64 generator seeded with `seed` (Steele, Lea and Flood, OOPSLA 2014),
 * top 53 bits scaled to [0, 1).  Paper: the urgency-estimation error study of Section 6.6. */
double pp_noise_factor(uint64_t seed, uint64_t frame_id, double eps);

/* Real-time trace replay (a load generator for serving measurements; the paper has no
 * counterpart).  Frame k arrives start + arrivals[k].t_us after the call begins (arrivals
 * sorted by t_us) and is submitted then, from the calling thread, with t_arrival = its
 * scheduled time and the first n_points points of clouds[cloud] (is_device_ptr: all clouds
 * device memory, borrowed for the call; else host memory, copied at submission).  Completed
 * frames are polled and released as they come; the call returns once every admitted frame has
 * completed, or PP_ETIMEDOUT timeout_us after the last arrival.  A frame the budget cannot
 * admit is counted as rejected (per chain) and not retried. */
typedef struct {
  double t_us;
  int32_t chain_id, cloud;
  int64_t n_points;
} pp_arrival;
typedef struct {
  uint64_t submitted, rejected, completed, dropped;
  uint64_t chain_rejected[PP_MAX_CHAINS];
  double wall_s;
  double submit_late_us_max, submit_late_us_mean;  /* submission behind its scheduled time */
} pp_replay_stats;
int pp_replay(pp_ctx* ctx, const pp_arrival* arrivals, int64_t n, const float* const* clouds,
              const int64_t* cloud_points, int32_t n_clouds, int32_t is_device_ptr, double timeout_us,
              pp_replay_stats* out);

/* ---------------------------------------------------------------------------------------- */
/* One release unit without the runtime: buffers for `max_batch` frames of one precision,    */
/* the whole front end as plain launches or one CUDA graph per batch size.  Paper: the GPU    */
/* segment of a 3D-perception chain (PointPillars, Section 6.1, Table 4), run as the work of   */
/* one release; the pipeline object itself has no counterpart in the paper.                  */
typedef struct pp_pipeline pp_pipeline;
/* Creates one unit for `precision` (PP_F32 / PP_BF16) from cfg's geometry, backbone, weights
 * and max_batch, tunes its conv tiles (cfg->autotune) and captures its graphs (cfg->use_graphs).
 * Section 6.1, Table 4 (the PointPillars segment).  Errors: PP_EINVAL, PP_ENOMEM, PP_EDEVICE. */
int pp_pipeline_create(const pp_config* cfg, int32_t precision, pp_pipeline** out);
/* frames: host array of n pointers to each frame's points (host or device memory, copied into
 * the unit's slots on `stream`); counts: host array of n point counts.  Enqueues everything on
 * `stream` and returns without waiting for it; a call first waits for the previous run on the
 * same pipeline to finish (the unit's per-launch table, in page-locked host memory, is read by
 * that run's first kernel).  Section 6.1, Table 4 (one release of the chain's GPU segment). */
int pp_pipeline_run(pp_pipeline* p, int32_t n, const float* const* frames,
                    const int32_t* counts, int32_t use_graph, void* stream);
/* Device pointer to block `block`'s output for frame slot i (padded NHWC) and its shape; pass
 * block = -1 for the number of pillars (int32 device pointer, dims unset), -2 for the head map
 * and -3 for the neck map (with a head configured; for the split FP32 form the value plane).
 * Pointers belong to the pipeline (valid until the next run or pp_pipeline_destroy).  No
 * counterpart in the paper (output access). */
int pp_pipeline_output(pp_pipeline* p, int32_t i, int32_t block, const void** dev,
                       int32_t* c, int32_t* h, int32_t* w);
/* Device bytes the pipeline holds; frees it.  No counterpart in the paper. */
size_t pp_pipeline_bytes(pp_pipeline* p);
int pp_pipeline_destroy(pp_pipeline* p);

/* ---------------------------------------------------------------------------------------- */
/* The release rule as a pure function (what the dispatcher calls on every decision), exported */
/* so that decisions can be replayed against an independent implementation.                  */
typedef struct {
  uint64_t frame_id;
  int32_t chain_id, precision;
  double t_arr_us, deadline_us, est_gpu_us, est_cpu_us;
  double util;                   /* GPU utilisation of the frame's kernels (delay exemption)  */
  double period_us;              /* its chain's period (PP_POLICY_LCUF)                       */
} pp_policy_frame;
typedef struct {
  int32_t chain_id;
  double ul;                     /* priority of an active unit when it was released           */
                                 /* (pp_policy_priority; urgency 1/us for PP_POLICY_URGENCY)  */
} pp_policy_active;
typedef struct {
  int32_t policy, max_batch, max_closed, num_pri, early_exit;
  double th_urgent, util_exempt;
  double eqdf_lambda;
} pp_policy_config;
enum { PP_DECIDE_NONE = 0, PP_DECIDE_RELEASE = 1, PP_DECIDE_WAIT = 2, PP_DECIDE_DELAY = 3 };
typedef struct {
  int32_t kind, level, n_frames, n_drops;
  uint64_t frames[8];            /* released frame ids (kind RELEASE), most urgent first     */
} pp_policy_decision;
/* One decision of the release rule at time t_us, as the dispatcher takes it: drop frames whose
 * slack is negative (early chain exit, Section 4.3; urgency policy only); WAIT while
 * closed_pending >= max_closed (batched launching with overlap, Section 4.4.5); order the rest
 * by least slack, i.e. highest UL of Eq. 2 (Section 4.2; the comparison policies of Section 6.4
 * by their own keys); DELAY while another chain's active unit is above TH_urgent and more
 * urgent than the head (Section 4.4.4); otherwise RELEASE the head and up to max_batch - 1
 * further frames of its precision at stream level 0 if UL > TH_urgent, else its normalised
 * rank among the active non-urgent units (Section 4.4.3).  Pure function of its arguments
 * (host arrays; nothing retained).
 * drops: caller array of drops_cap entries receiving the ids of frames to drop (early exit);
 * n_drops counts them all even if more than drops_cap.  PP_EINVAL for a bad argument. */
int pp_policy_decide(const pp_policy_config* cfg, double t_us, const pp_policy_frame* ready,
                     int32_t n_ready, const pp_policy_active* active, int32_t n_active,
                     int32_t closed_pending, pp_policy_decision* out, uint64_t* drops,
                     int32_t drops_cap);
/* A frame's priority under cfg->policy at time t (higher = released first; Eq. 2 and the
 * comparison policies of Section 6.4): URGENCY: UL = 1 /
 * slack (-inf for slack <= 0); EDF: -deadline; SJF: -(est_gpu + est_cpu); HRRN: (t - t_arr +
 * e) / e with e = est_gpu + est_cpu (+inf when e <= 0); LCUF: -(e / period) (-inf when the
 * period is not positive); SAEDF: -deadline, less 1e15 us when slack < 0; EQDF: -(deadline -
 * eqdf_lambda * e); FIFO: -t_arr.  Stream levels rank active units by this value. */
double pp_policy_priority(const pp_policy_config* cfg, double t_us, const pp_policy_frame* frame);

/* Decision log (pp_config.decision_log > 0; the paper has no counterpart: it lets every release
 * decision a serving run took be replayed against an independent restatement of the rule).
 * Record k holds the inputs the dispatcher passed to pp_policy_decide -- the time, the rule's
 * configuration as it stood (th_urgent as calibrated), the ready frames as the rule saw them
 * (estimates with any estimate noise applied), the active units and the closed batches pending
 * -- and the decision it returned.  Its ready frames are ready[ready_off .. ready_off +
 * n_ready), its active units active[active_off .. + n_active), its drops drops[drops_off ..
 * + decision.n_drops).  launched: for a RELEASE, 1 if the unit was launched, 0 if no unit of
 * that precision was free (the frames stayed ready). */
typedef struct {
  double t_us;
  pp_policy_config cfg;
  int32_t closed_pending, n_ready, n_active, launched;
  int64_t ready_off, active_off, drops_off;
  pp_policy_decision decision;
} pp_decision_record;
/* Copies the log.  With recs == NULL only the sizes are written (n_recs, n_ready, n_active,
 * n_drops; each pointer may be NULL); otherwise every array must hold the sizes a previous
 * query returned (max_* entries; PP_EINVAL if one is too small) and is filled.  The log stops
 * growing at pp_config.decision_log records; reading it does not clear it. */
int pp_decision_log(pp_ctx* ctx, pp_decision_record* recs, int32_t max_recs, pp_policy_frame* ready,
                    int64_t max_ready, pp_policy_active* active, int64_t max_active, uint64_t* drops,
                    int64_t max_drops, int32_t* n_recs, int64_t* n_ready, int64_t* n_active,
                    int64_t* n_drops);

#ifdef __cplusplus
}
#endif
#endif /* PP_H_ */
