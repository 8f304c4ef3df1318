/*
 * dfb.h - C ABI of a single-GPU Distributed FrameBuffer compositing library.
 *
 * The operations follow Usher et al., "Scalable Ray Tracing Using the
 * Distributed FrameBuffer" (EuroVis 2019):
 *   - a frame is bracketed by begin/end and fed tile by tile with setTile
 *     (Sec. 3.1, the tile processing pipeline);
 *   - a tile carries RGBA colour and depth for TxT pixels (Listing 1, Tile);
 *   - per tile, a dependency tree of generations tells the owner how many
 *     inputs to wait for (Sec. 3.1.1, Listing 3: a generation-0 background
 *     tile declares the number of generation-1 children);
 *   - the AlphaBlend tile operation orders each pixel's fragments by depth
 *     before combining them (Sec. 4.2, Listing 4); with a rank-order tree the
 *     tiles are combined in list order instead (Sec. 4.2);
 *   - progressive refinement keeps accumulation and variance tiles
 *     (Listing 1, TileOperation; Sec. 4.1.1 uses the variance to steer work);
 *   - the finished tile is converted to the RGBA8 or RGBAF32 display format
 *     (Sec. 3.1).
 * The paper's ranks become fragment producers in one process; its per-tile
 * owners become work items of CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *   - Return value: DFB_OK (0) or a negative DFB_ERR_* code.  No C++
 *     exception crosses this interface: a host allocation that fails inside
 *     a call returns DFB_ERR_OOM (an open frame may then hold part of that
 *     call's tiles: begin the frame again).  dfb_error_string() names a
 *     code.
 *   - Pixels: a fragment tile is T*T pixels, row-major inside the tile
 *     (pixel p = y*T + x).  Frames are row-major images W*H.  Tiles are
 *     numbered row-major: tile = ty * ceil(W/T) + tx.  Pixels of a submitted
 *     tile that fall outside the frame (ragged right/bottom tiles) are ignored.
 *   - Colour is premultiplied RGBA.  Depth is FP32 in every storage mode;
 *     NaN depth is read as +inf and -0.0 as +0.0.  An empty fragment pixel is
 *     RGBA 0 with depth +inf.
 *   - Ownership: the caller owns every pointer it passes.  A device pointer
 *     given to a submit call is borrowed until the work of the dfb_end_frame
 *     call that consumes it has finished on its stream.  A host pointer is
 *     copied before the submit call returns, unless it is submitted as
 *     DFB_PTR_HOST_BORROWED: then it is borrowed like a device pointer.
 *     The handle owns the resident framebuffers (colour, accumulation,
 *     variance, RGBA8).
 *   - Threads: a handle must not be used by two threads at once.
 *   - Device: a handle lives on the device that was current when it first
 *     allocated device memory (at creation, or at its first frame with
 *     DFB_FLAG_DEFER_ALLOC).  Calls that enqueue device work with another
 *     device current return DFB_ERR_STATE.
 */
#ifndef DFB_H
#define DFB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DFB_API __attribute__((visibility("default")))
#else
#define DFB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dfb_ctx* dfb_handle;

/* Tile operation (compositing mode). */
enum dfb_mode {
  DFB_BLEND_DEPTH = 0,   /* per-pixel sort by (depth, key, submit index), then
                            front-to-back "over" (Sec. 4.2, Listing 4)        */
  DFB_BLEND_ORDERED = 1, /* "over" in (key, submit index) order for every
                            pixel: the rank-order list tree of Sec. 4.2       */
  DFB_ZCOMPOSITE = 2,    /* nearest (depth, key, submit index) fragment wins,
                            RGBA copied unchanged (depth compositing, Sec. 2.1)*/
  DFB_AVERAGE = 3        /* per-pixel mean of the tile's fragments, equal
                            weights, depth ignored: redundantly rendered tiles
                            of the image-parallel renderer (Sec. 4.1.1)       */
};

/* Pixel operation run on the finished value just before the RGBA8 display
   conversion (Sec. 3.1.2; the paper leaves the formula to the user).  All act
   on premultiplied RGB with alpha unchanged; e is the operation's exposure. */
enum dfb_pixel_op {
  DFB_PIXELOP_NONE = 0,
  DFB_PIXELOP_EXPOSURE = 1,  /* rgb -> e * rgb                                */
  DFB_PIXELOP_REINHARD = 2,  /* rgb -> e*rgb / (1 + e*rgb), per channel        */
  DFB_PIXELOP_CURVE = 3      /* rgb -> the user's tone curve of each channel
                                at e*rgb (dfb_set_pixel_curve)                */
};

/* Storage type of the submitted fragment RGBA (depth is always FP32). */
enum dfb_dtype {   /* every RGBA tile and depth plane must be 16-byte aligned */
  DFB_F32 = 0,     /* 4 x float32 per pixel                                 */
  DFB_F16 = 1,     /* 4 x IEEE binary16 per pixel                           */
  DFB_BF16 = 2,    /* 4 x bfloat16 per pixel                                */
  DFB_FP8E4M3 = 3  /* 4 x e4m3 codes per pixel; value =
                      decode(code) * the fragment's FP32 scale               */
};

enum dfb_status {
  DFB_OK = 0,
  DFB_ERR_INVALID_ARG = -1, /* bad size, null or misaligned pointer, NaN key  */
  DFB_ERR_TILE_RANGE = -2,  /* tile id outside [0, tiles)                      */
  DFB_ERR_STATE = -3,       /* call not allowed in the handle's current state  */
  DFB_ERR_INCOMPLETE = -4,  /* a tile's dependency tree is not complete         */
  DFB_ERR_OOM = -5,         /* device or pinned allocation failed               */
  DFB_ERR_TIMEOUT = -6,     /* a device-side wait gave up                        */
  DFB_ERR_CUDA = -7,        /* a CUDA call failed (including: no device)         */
  DFB_ERR_CAPACITY = -8,    /* request larger than dfb_composite_noalloc's fixed
                               scratch (see its limits below)                   */
  DFB_ERR_CHECK = -9        /* a device-side bounds check of the checked build
                               (libdfb_checked.so) failed; the access was
                               skipped and the launch ended early             */
};

/* Configuration flags. */
#define DFB_FLAG_ACCUMULATE 1u  /* keep accumulation + variance buffers        */
#define DFB_FLAG_WRITE_COLOR 2u /* write the float RGBA frame (RGBAF32 format)  */
#define DFB_FLAG_PACK_RGBA8 4u  /* write the sRGB RGBA8 frame                   */
#define DFB_FLAG_DEFER_ALLOC 8u /* allocate device memory at the first
                                   dfb_end_frame instead of at creation         */
#define DFB_FLAGS_DEFAULT (DFB_FLAG_ACCUMULATE | DFB_FLAG_WRITE_COLOR | DFB_FLAG_PACK_RGBA8)

/* Where the pointers of a bulk submit live. */
#define DFB_PTR_AUTO 0   /* ask the CUDA runtime for each pointer */
#define DFB_PTR_DEVICE 1 /* all device (or managed) memory         */
#define DFB_PTR_HOST 2   /* all host memory (pageable or pinned), copied to the
                            device before the submit call returns           */
#define DFB_PTR_HOST_BORROWED 3 /* host memory copied to the device
                            asynchronously: like a device pointer, it is
                            borrowed until the work of the dfb_end_frame call
                            that consumes it has finished (dfb_sync, or the
                            stream), and must not change before            */

typedef struct dfb_config {
  int width;         /* frame width in pixels, >= 1                          */
  int height;        /* frame height in pixels, >= 1                         */
  int tile_size;     /* T: a power of two in [4, 256]                        */
  int mode;          /* enum dfb_mode                                        */
  int dtype;         /* enum dfb_dtype                                       */
  unsigned flags;    /* DFB_FLAG_*                                           */
  int kahan_after;   /* accumulated frames after which the running sum is
                        Kahan-compensated; <= 0 selects 256                  */
  int max_fragments; /* initial record capacity hint; <= 0 selects 4096      */
} dfb_config;

/* One submitted tile (the paper's Tile of Listing 1, data + tree fields). */
typedef struct dfb_tile_desc {
  int tile_id;        /* destination tile                                    */
  float order_key;    /* e.g. distance from the eye to the brick centre      */
  const void* rgba;   /* T*T*4 values of the handle's dtype                  */
  const float* depth; /* T*T FP32 depths                                     */
  float scale;        /* FP8 dequantisation scale (> 0, finite); else ignored */
  int generation;     /* >= 1; rendered data tiles are generation 1          */
  int children;       /* tiles this one adds to generation+1 (>= 0)          */
} dfb_tile_desc;

typedef struct dfb_frame_stats {
  int64_t fragments;         /* tiles composited by the last frame            */
  int64_t fragment_pixels;   /* sum over fragments of in-frame pixels          */
  int64_t frame_pixels;      /* W * H                                          */
  int64_t fragment_bytes;    /* algorithmic bytes of fragment data read        */
  int64_t state_bytes;       /* algorithmic bytes of framebuffer state moved   */
  int32_t accumulated;       /* frames in the accumulation (1 after a reset)   */
  int32_t tiles;             /* tiles in the frame                             */
  int64_t kernel_launches;   /* kernels this handle has launched in total      */
} dfb_frame_stats;

/* Create a framebuffer with DFB_FLAGS_DEFAULT and FP32 storage.  Sizes: at
   most 2^31 pixels, and at most 2^32 pixels in its whole tiles
   (ceil(W/T) * ceil(H/T) * T * T).
   Errors: INVALID_ARG (sizes, mode, tile size), OOM, CUDA (no device). */
DFB_API int dfb_create(int width, int height, int tile_size, int mode, dfb_handle* out);

/* Create a framebuffer from a full configuration.  Same errors. */
DFB_API int dfb_create_ex(const dfb_config* cfg, dfb_handle* out);

/* Release the handle and its device memory (synchronises its last frame).
   A null handle is accepted and ignored.  Always returns DFB_OK. */
DFB_API int dfb_destroy(dfb_handle h);

/* Background colour (unpremultiplied RGB and coverage A): the generation-0
   background tile of Sec. 4.2, blended behind every pixel in the blend modes
   and DFB_AVERAGE and shown by empty tiles in DFB_ZCOMPOSITE.  Default
   (0,0,0,0); applies from the next dfb_end_frame.  Errors: INVALID_ARG
   (null handle, a component not finite). */
DFB_API int dfb_set_background(dfb_handle h, float r, float g, float b, float a);

/* Pixel operation of the RGBA8 output (enum dfb_pixel_op) with its exposure,
   from the next dfb_end_frame on.  The colour, accumulation and variance
   buffers are not affected.  Errors: INVALID_ARG (unknown op, exposure not
   finite or negative), STATE (DFB_PIXELOP_CURVE before any
   dfb_set_pixel_curve on this handle). */
DFB_API int dfb_set_pixel_op(dfb_handle h, int op, float exposure);

/* Load a user tone curve per colour channel and select DFB_PIXELOP_CURVE
   (the exposure set last is kept): the user-supplied pixel operation of
   Sec. 3.1.2, fused into the RGBA8 pack.
   curves: host array of 3*n floats, channel-major (n samples of R, then G,
   then B); sample j of a channel is the curve's value at
   x_j = x_max * j / (n - 1).  The curve is piecewise linear between samples;
   the input x = e * rgb is clamped to [0, x_max] first (NaN reads as 0).
   The result is a linear value that the sRGB pack then encodes.
   The samples are copied into a device buffer of the handle (4096 samples
   per channel at most) before the call returns; the call first waits for the
   handle's frames in flight.  A CUDA graph captured from this handle reads
   that buffer when it runs, with the n and x_max of its capture; the caller
   must not load a curve while such a replay is in flight.
   Errors: INVALID_ARG (null curves, n outside [2, 4096], x_max not finite or
   <= 0, a sample not finite), STATE (another device is current than the
   handle's or the curve's), OOM, CUDA. */
DFB_API int dfb_set_pixel_curve(dfb_handle h, const float* curves, int n, float x_max);

/* Begin a frame (Sec. 3.1).  accumulate = 0 restarts the progressive
   accumulation with this frame; non-zero adds this frame to it.
   Errors: STATE if a frame is already open. */
DFB_API int dfb_begin_frame(dfb_handle h, int accumulate);

/* Declare the generation-0 tile of a tile's dependency tree with n_children
   generation-1 inputs (Sec. 3.1.1, Listing 3).  Tiles with no declaration
   composite whatever arrives.  Errors: STATE, TILE_RANGE, INVALID_ARG (n<0),
   STATE if the tile already has a declaration this frame. */
DFB_API int dfb_set_tile_children(dfb_handle h, int tile_id, int n_children);

/* setTile for one rendered generation-1 tile (Sec. 3.1).  rgba/depth may be
   host or device pointers.  Errors: STATE (no open frame), TILE_RANGE,
   INVALID_ARG (NaN key, null/misaligned pointer, or an FP8 handle, whose
   tiles need a scale: use dfb_submit_tile_ex), OOM, CUDA. */
DFB_API int dfb_submit_tile(dfb_handle h, int tile_id, float order_key, const void* rgba,
                    const float* depth);

/* setTile with the tree fields and the FP8 scale.  Same errors. */
DFB_API int dfb_submit_tile_ex(dfb_handle h, const dfb_tile_desc* tile);

/* Bulk setTile of n generation-1 tiles (index i is submitted before i+1).
   Arrays are host arrays of length n; scales may be NULL unless the dtype is
   FP8.  `where` is a DFB_PTR_* hint.  The whole call is validated first and
   nothing is submitted if any entry is invalid; the error of the first bad
   entry is returned. */
DFB_API int dfb_submit_tiles(dfb_handle h, int n, const int* tile_ids, const float* order_keys,
                     const void* const* rgba, const float* const* depth,
                     const float* scales, int where);

/* Bulk setTile with the tree fields and scales: tiles[0..n) in order, with the
   same all-or-nothing validation and `where` hint as dfb_submit_tiles.
   Errors: as dfb_submit_tiles (STATE, TILE_RANGE, INVALID_ARG, OOM, CUDA). */
DFB_API int dfb_submit_tiles_ex(dfb_handle h, int n, const dfb_tile_desc* tiles, int where);

/* End the frame: check every declared dependency tree (INCOMPLETE if a
   generation received more or fewer tiles than its parents declared; the
   frame then stays open so the missing tiles can still be submitted), then
   enqueue the compositing, accumulation, variance and pack kernels on
   `stream` (a cudaStream_t; NULL = the legacy default stream) and return
   without waiting.  Refused with STATE on a stream that is being captured
   into a CUDA graph (the captured record upload would replay stale records;
   dfb_graph_create captures frames correctly).
   Errors: STATE, INCOMPLETE, OOM, CUDA. */
DFB_API int dfb_end_frame(dfb_handle h, void* stream);

/* ---- Prepared submissions ------------------------------------------------------
   A producer that renders into the same tile buffers every frame (the
   progressive-refinement passes of Sec. 4.1, the per-rank brick buffers of
   Sec. 4.2) submits the same list each frame.  A dfb_tileset is that list --
   the arguments of one dfb_submit_tiles call with device pointers --
   validated once and kept as ready records, so submitting it again costs one
   copy of 32 bytes per tile.  The set borrows the device pointers: they must
   stay valid (their contents may change) while any frame that used the set
   can still run. */
typedef struct dfb_tileset_t* dfb_tileset;

/* Validate n generation-1 tiles against the geometry and dtype of `h` (as
   dfb_submit_tiles with DFB_PTR_DEVICE does) and keep them as a set usable
   with every handle of the same width, height, tile size and dtype.  Arrays
   are host arrays of length n (n >= 0); scales may be NULL unless the dtype
   is FP8.  Errors: INVALID_ARG, TILE_RANGE, OOM. */
DFB_API int dfb_tileset_create(dfb_handle h, int n, const int* tile_ids, const float* order_keys,
                               const void* const* rgba, const float* const* depth,
                               const float* scales, dfb_tileset* out);
DFB_API int dfb_tileset_destroy(dfb_tileset s);

/* Submit a prepared set into the open frame of `h`: the same records, in the
   same order, as the dfb_submit_tiles call it was made from.  Errors:
   INVALID_ARG (null, or a set made for another geometry or dtype), STATE. */
DFB_API int dfb_submit_tileset(dfb_handle h, dfb_tileset s);

/* One step of a compositing server: for every i, begin a frame on hs[i]
   (accumulating onto its previous frames if accumulate[i] != 0; accumulate
   may be NULL = no accumulation), submit sets[i], then end all frames with
   one batched launch on `stream` (dfb_end_frames).  Everything is validated
   before any frame is begun: handles distinct and not inside a frame, sets
   matching their handles, one dtype, a stream that is not being captured.
   If the launch itself fails (OOM, CUDA) the frames stay open, as after a
   failed dfb_end_frames.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
DFB_API int dfb_run_frames(const dfb_handle* hs, const dfb_tileset* sets, const int* accumulate,
                           int n, void* stream);

/* Composite the open frames of several handles with one persistent launch on
   `stream`: the batched form of dfb_end_frame.  Every handle is validated
   first; on any error nothing is launched and the first error is returned.
   Handles must be distinct. */
DFB_API int dfb_end_frames(const dfb_handle* hs, int n, void* stream);

/* Wait for the last frame's work.  Errors: CUDA, TIMEOUT (a device queue
   gave up; the frame's outputs are then undefined). */
DFB_API int dfb_sync(dfb_handle h);

/* Copy the finished frame as W*H*4 floats (RGBAF32 display format).  `out`
   may be host memory (the call waits) or device memory (the copy is ordered
   after the last frame on its stream).  Errors: STATE if no frame has been
   composited or the colour buffer is disabled, CUDA. */
DFB_API int dfb_read_color(dfb_handle h, float* out);

/* Copy the normalised accumulation (sum of frames / frame count), W*H*4
   floats.  Errors: STATE if accumulation is disabled or empty, CUDA. */
DFB_API int dfb_read_accum(dfb_handle h, float* out);

/* Copy the per-pixel sample variance (W*H*4 floats, ddof = 1, 0 after one
   frame) and/or the per-tile variance (tiles floats: mean over in-frame
   pixels of the RGB variances).  Either pointer may be NULL.  Errors:
   INVALID_ARG (null handle), STATE (accumulation disabled or no frame yet),
   OOM, CUDA, TIMEOUT / CHECK (reported by the last frame's launch). */
DFB_API int dfb_read_variance(dfb_handle h, float* per_pixel, float* per_tile);

/* Copy the sRGB RGBA8 frame, W*H uint32 with bytes R,G,B,A in memory order
   (host or device `out`; a host copy waits for the frame).  Errors:
   INVALID_ARG (null), STATE (packing disabled or no frame yet), CUDA,
   TIMEOUT / CHECK (reported by the last frame's launch). */
DFB_API int dfb_read_rgba8(dfb_handle h, uint32_t* out);

/* Statistics of the last composited frame.  Errors: INVALID_ARG (null). */
DFB_API int dfb_get_stats(dfb_handle h, dfb_frame_stats* out);

/* Tile grid of the handle.  Errors: INVALID_ARG (null). */
DFB_API int dfb_get_tiles(dfb_handle h, int* tiles_x, int* tiles_y);

/* Checkpoint of the progressive state: running sum, Kahan compensation and
   M2 (each W*H*4 floats, host or device) and the frame count.  Load restores
   it so accumulation resumes bit-identically.  Errors: INVALID_ARG (null
   pointer), STATE (accumulation disabled or no frame yet), OOM, CUDA. */
DFB_API int dfb_save_accum(dfb_handle h, float* sum, float* comp, float* m2, int* frames);
DFB_API int dfb_load_accum(dfb_handle h, const float* sum, const float* comp, const float* m2,
                   int frames);

/* Producer-side conversion of FP32 fragment tiles (device pointers) to a
   storage dtype, on `stream`.  n_tiles tiles of tile_pixels pixels each.
   DFB_F16/DFB_BF16: round to nearest even.  DFB_FP8E4M3: per tile,
   scale = amax/448 (1 if the tile is all zero), code = e4m3(x / scale) with
   round-to-nearest-even and saturation; scales (device, n_tiles floats)
   receives the scales.  Errors: INVALID_ARG, CUDA. */
DFB_API int dfb_convert_tiles(const float* src, void* dst, float* scales, int n_tiles,
                      int tile_pixels, int dtype, void* stream);

/* Per-stage device timing (tracing).  While enabled, every dfb_end_frame /
   dfb_end_frames call records CUDA events around its bucketing kernel and its
   persistent composite kernel on their streams (the re-do and per-tile
   variance kernels that follow the composite are not included).  The events
   sit between kernels that otherwise start while the kernel before them
   drains (programmatic launches), so a frame takes a few microseconds longer
   while timing is on.  dfb_read_timing waits for the recorded events, adds
   them up since the last reset and, if reset != 0, starts a new sum.  For
   dfb_end_frames the batch is timed on its first handle.  Errors:
   INVALID_ARG, CUDA. */
typedef struct dfb_timing {
  int32_t launches;     /* end-of-frame launches timed                        */
  float bucket_ms;      /* total time of the bucketing kernel (K1)            */
  float composite_ms;   /* total time of the composite kernel (K2/K3 + K4)    */
} dfb_timing;
DFB_API int dfb_set_timing(dfb_handle h, int enable);
DFB_API int dfb_read_timing(dfb_handle h, dfb_timing* out, int reset);

/* Composite one frame in a single call that allocates no memory at all.
   The paper has no counterpart: it is an interface for callers that must not
   call cudaMalloc -- e.g. an in-situ simulation or renderer that reserves the
   whole GPU and hands out memory only from its own pool, or real-time code in
   which a cudaMalloc/cudaFree could synchronise the device and miss a frame
   deadline.  The handle-based path above allocates framebuffers and scratch,
   so such callers use this instead.
   Inputs are those of dfb_submit_tiles (host arrays of length n; rgba/depth
   are DEVICE pointers to T*T-pixel tiles of `dtype`; scales only for FP8),
   plus an optional unpremultiplied background (4 floats, NULL = 0).  Outputs
   are caller-owned DEVICE buffers: color_out (W*H*4 floats) and/or rgba8_out
   (W*H uint32, sRGB of the frame colour); either may be NULL, not both.
   There is no accumulation or variance (those need resident state).
   Scratch: a fixed device array of about 15 MB inside the library, held by
   every GPU that loads it until the process exits.  Limits: n <= 65536
   fragment tiles and ceil(W/T)*ceil(H/T) <= 16384 tiles; larger requests
   return DFB_ERR_CAPACITY before any GPU work.  The first call on a device
   looks up the array's device address (and uploads the sRGB table) with that
   device current.  All calls share the one array, which keeps the previous
   call's contents (the call clears what must start at zero): calls whose GPU
   work overlaps -- on two streams, or from two threads -- race and must be
   serialised by the caller.
   The call is synchronous: it copies the host arrays, queues the work on
   `stream`, waits for it and returns the device status of the launch, so a
   return of DFB_OK means the outputs are complete.  It copies from pageable
   host memory and waits on the stream, so it must never be made on a stream
   that is being captured into a CUDA graph (refused with DFB_ERR_STATE
   before the stream is touched).  Errors: INVALID_ARG (sizes, NaN key, null
   or misaligned pointer, an output or input tile that is not device or
   managed memory -- for inputs laid out back to back, the first and last
   tile of each run are checked), TILE_RANGE, CAPACITY, STATE (capturing
   stream), TIMEOUT (a wait inside the kernels ran out; the outputs are
   incomplete), CHECK (checked build: a device-side bounds check failed),
   OOM (host), CUDA. */
DFB_API int dfb_composite_noalloc(int width, int height, int tile_size, int mode, int dtype,
                                  int n, const int* tile_ids, const float* order_keys,
                                  const void* const* rgba, const float* const* depth,
                                  const float* scales, const float* background,
                                  float* color_out, uint32_t* rgba8_out, void* stream);

/* Failure detection of dfb_composite_noalloc, for tests of its timeout path
   (process-wide settings, like the call's scratch).  dfb_noalloc_set_wait_limit
   bounds every wait inside its kernels (default 2 s); dfb_noalloc_inject_stall
   makes the next call leave work item `item` unfilled (-1: off), so that its
   consumers' wait runs out after the limit and the call returns
   DFB_ERR_TIMEOUT with incomplete outputs; the setting is used up by that
   call.  Errors: INVALID_ARG (a limit <= 0 or > 3600 s, item < -1). */
DFB_API int dfb_noalloc_set_wait_limit(double seconds);
DFB_API int dfb_noalloc_inject_stall(int item);

/* ---- Batched frames replayed from a CUDA graph ------------------------------
   A dfb_graph holds the device work of compositing the open frames of several
   handles -- record upload done once, then per launch: the bucketing kernel
   and ONE persistent composite launch over every work item of every frame
   (plus the re-do and per-tile variance kernels) -- captured in a CUDA
   graph.  Each launch
   re-reads the fragment tiles through the same device pointers, so producers
   may rewrite their tiles in place between launches.  Frame arguments are
   frozen at creation: an accumulating handle keeps the frame count it had
   (use dfb_end_frame for progressive accumulation).  The handles must stay
   alive and unused by other calls while the graph exists; results are read
   with the usual dfb_read_* calls after a launch. */
typedef struct dfb_graph_t* dfb_graph;

/* Capture the open frames of hs[0..n) (all of one dtype, distinct handles).
   Their trees are checked as in dfb_end_frames and the frames are ended.
   Errors: INVALID_ARG, STATE, INCOMPLETE, OOM, CUDA. */
DFB_API int dfb_graph_create(const dfb_handle* hs, int n, dfb_graph* out);

/* Replay the captured work on `stream`.  Errors: INVALID_ARG (null or
   failed graph), CUDA. */
DFB_API int dfb_graph_launch(dfb_graph g, void* stream);

/* Re-capture with another composite launch shape (see dfb_set_tuning).
   Errors: INVALID_ARG (a shape not in the list), CUDA (the shape does not fit
   the device). */
DFB_API int dfb_graph_set_tuning(dfb_graph g, int ring_kb, int ctas_per_sm, int groups);

/* Autotuner: time `reps` replays of each candidate launch shape (ring size =
   pipeline depth, CTAs per SM, consumer groups per CTA) on `stream`, keep the
   fastest, and report it (any pointer may be NULL).  The graph's handles get
   the same tuning for their later dfb_end_frame calls.  Errors: INVALID_ARG,
   CUDA. */
DFB_API int dfb_graph_autotune(dfb_graph g, void* stream, int reps, int* ring_kb,
                               int* ctas_per_sm, int* groups, float* best_ms);

/* Free the graph and its buffers (waits for its last launch).  A null graph
   is accepted.  Always returns DFB_OK. */
DFB_API int dfb_graph_destroy(dfb_graph g);

/* Launch shape of this handle's composite kernel: shared-memory ring size per
   CTA in KB (how many work items are in flight), persistent CTAs per SM, and
   consumer groups per CTA (work items composited at once by one CTA).  The
   shapes built are (groups, CTAs per SM) = (1, 2), (2, 2), (1, 3), (2, 1)
   and (3, 1).  0, 0, 0 restores the library default, chosen per launch:
   2 CTAs per SM with one group for FP32 and for frames of 5 or more
   fragment tiles per image tile, else 3 CTAs per SM.  A ring larger
   than the CTAs can share is clamped at launch; one too small for the
   largest work item of the dtype makes the launch fail with DFB_ERR_CUDA.
   Errors: INVALID_ARG (a shape not in the list). */
DFB_API int dfb_set_tuning(dfb_handle h, int ring_kb, int ctas_per_sm, int groups);

/* Bound on every wait inside the composite kernel (default 2 s).  A wait
   that runs out makes the kernel give up, and the next dfb_sync (or host
   read) returns DFB_ERR_TIMEOUT.  Errors: INVALID_ARG (<= 0 or > 3600). */
DFB_API int dfb_set_wait_limit(dfb_handle h, double seconds);

/* Fault injection for tests of the timeout path: the next end-of-frame
   launch of this handle never fills work item `item` (-1: off), so its
   consumers' wait runs out after the wait limit.  Errors: INVALID_ARG. */
DFB_API int dfb_inject_stall(dfb_handle h, int item);

/* Human-readable name of a status code (static storage). */
DFB_API const char* dfb_error_string(int status);

/* Library version, major*10000 + minor*100 + patch. */
DFB_API int dfb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DFB_H */
