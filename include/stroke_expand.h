/*
 * stroke_expand.h -- C ABI of the GB300 stroke-expansion library.
 *
 * Implements the data-parallel stroke expansion of R. Levien and A. Uguray,
 * "GPU-friendly Stroke Expansion" (arXiv 2405.00127): stroked paths of line
 * and cubic Bezier segments, with width, join, cap and optional dash style,
 * become strongly correct outlines made of line or circular-arc segments.
 *
 * The library has two halves:
 *   - a host encoder (the paper's CPU step, Section 8.2) that turns SVG-style
 *     verbs into the tag / point / style streams of Table 1;
 *   - device expansion on one GPU: a segmented tag-monoid scan, a count pass,
 *     an exclusive scan of the counts and a write pass (Sections 7 and 8,
 *     Algorithms 1 and 2), all in the library's own CUDA kernels;
 *   - for scenes with dash patterns, a device dash pass before the expansion
 *     (SVG dash semantics; the paper dashes on the CPU, Section 9.3): FP32 arc
 *     lengths, a compensated segmented scan per subpath, and a rewrite of every
 *     "on" interval into an open subpath of its own.
 *
 * Conventions
 *   - Every function returns an se_status; nothing throws across the ABI.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the context's device.  The caller owns every buffer it
 *     passes in; the library owns the context and its workspace.
 *   - Device calls are asynchronous on the context's stream unless stated.
 *   - Coordinates and all device arithmetic are IEEE FP32 (Section 1: the
 *     method must stay robust in 32-bit floating point).
 */
#ifndef STROKE_EXPAND_H
#define STROKE_EXPAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum se_status {
    SE_OK = 0,
    SE_ERR_INVALID_ARG = 1,    /* a NULL or out-of-range argument */
    SE_ERR_INVALID_INPUT = 2,  /* malformed verbs/tags, non-finite coordinates, bad style */
    SE_ERR_OOM = 3,            /* device allocation failed */
    SE_ERR_LIMIT = 4,          /* a per-range primitive count reached SE_MAX_RANGE_COUNT and was clamped */
    SE_ERR_CAPACITY = 5,       /* the caller's outline buffers are too small; nothing was written */
    SE_ERR_CUDA = 6,           /* a CUDA runtime call failed (see se_ctx_last_error) */
    SE_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
    SE_ERR_WORKSPACE = 8,      /* the context's piece workspace was too small for this scene: nothing
                                  was written; one se_count of the scene sizes it */
    SE_ERR_BUDGET = 9,         /* a served request's outline alone is larger than the server's HBM budget */
} se_status;

/* SVG-style verbs (Section 8.1) and the points each consumes */
enum {
    SE_VERB_MOVE = 0 /* 1 point */, SE_VERB_LINE = 1 /* 1 */, SE_VERB_CUBIC = 2 /* 3 */, SE_VERB_CLOSE = 3 /* 0 */,
    SE_VERB_QUAD = 4 /* 2: a quadratic Bezier, degree-elevated on the device (Section 8.1) */
};
enum { SE_JOIN_BEVEL = 0, SE_JOIN_MITER = 1, SE_JOIN_ROUND = 2 };
enum { SE_CAP_BUTT = 0, SE_CAP_SQUARE = 1, SE_CAP_ROUND = 2 };
enum { SE_OUT_LINES = 0, SE_OUT_ARCS = 1 };

/* Path tag bits (Table 1).  Bit 7 is this library's extension: it marks the
 * subpath-end tag (the stroke cap marker) of a closed subpath.
 *
 * The path data stream is a sequence of 32-bit words.  A tag with the F32 bit
 * has 32-bit coordinates, two words per point (float x, float y); without it,
 * 16-bit integer coordinates, one word per point (x in the low half, y in the
 * high half, two's complement).  Every tag of a subpath has the same width.
 * A tag's first point is the previous tag's last (the segments of a subpath
 * share their boundary points), except on the first tag of a subpath (the
 * first tag of the stream or one after a subpath-end or path bit), whose
 * first point is the subpath's start.  So each tag adds to the stream
 * (coordinate count + 1 if it starts a subpath) x (2 if F32 else 1) words; an
 * empty tag (count 0) adds none.  (Table 1 counts the start point on the end
 * tag of the previous subpath instead; counting it on the subpath's own first
 * tag keeps all of a subpath's points at its own width, and gives the same
 * stream when every tag is 32-bit.) */
#define SE_TAG_COUNT_MASK   0x03u  /* coordinate count: 1 line, 2 quadratic (the cap marker when the
                                      subpath-end bit is set), 3 cubic; 0 = empty path */
#define SE_TAG_SUBPATH_END  0x04u
#define SE_TAG_F32          0x08u  /* 32-bit coordinates (clear: 16-bit integer coordinates) */
#define SE_TAG_PATH         0x10u  /* last tag of a path */
#define SE_TAG_TRANSFORM    0x20u  /* this tag starts a new transform-stream entry (tags before the
                                      first such tag use the identity) */
#define SE_TAG_STYLE        0x40u  /* this tag starts a new style-stream entry */
#define SE_TAG_CLOSED       0x80u

/* Largest number of primitives one flattening range may produce. */
#define SE_MAX_RANGE_COUNT  65536u

/* Style of a path (24 bytes).  For a stroke: half_width > 0; miter_limit >= 1
 * is the SVG miter ratio limit; dash_count == 0 means a solid stroke, otherwise
 * the dash pattern is dashes[dash_first .. dash_first + dash_count) (SVG
 * semantics, repeated twice when odd) starting at dash_offset.
 * fill != 0 makes the path a fill (the fill branch of Algorithm 1): every
 * subpath is closed (with a closing line where its end differs from its
 * start) and its segments are flattened at offset 0 in their own direction;
 * width, joins, caps and dashes do not apply. */
typedef struct se_style {
    float half_width;
    float miter_limit;
    uint8_t join;
    uint8_t cap;
    uint8_t fill;
    uint8_t reserved;
    uint32_t dash_first;
    uint32_t dash_count;
    float dash_offset;
} se_style;

/* Expansion parameters.  tol is the output tolerance (device units).  The
 * cubic -> Euler-spiral fit is accepted at tol * fit_frac and parallel curves
 * are flattened at tol * flat_frac (the paper leaves the split open; the
 * library's defaults are 0.2 and 1.0). */
typedef struct se_params {
    float tol;
    float fit_frac;
    float flat_frac;
    uint32_t out_kind;     /* SE_OUT_LINES or SE_OUT_ARCS */
    uint32_t refine;       /* 0: fast; 1: refined line output (Section 4.2): counts from the
                            * exact integral of Section 4.1, vertices by two Newton steps
                            * from the approximation's inverse.  Fills and arc output are
                            * the same in both modes. */
} se_params;

/* ------------------------------------------------------------------------ */
/* Host encoder (Section 8.2, Table 1)                                      */
/* ------------------------------------------------------------------------ */

/* Sizes of the encoding of a verb scene.
 *   verbs[n_verbs]            host; SE_VERB_* codes; every path starts with MOVE
 *   pts[2 * n_pts]            host; x, y pairs consumed by the verbs in order
 *   path_verb_off[n_paths+1]  host; path p owns verbs [off[p], off[p+1])
 *   styles[n_paths]           host, may be NULL (every path a stroke): only
 *                             the fill flag changes the sizes
 *   coord16[n_paths]          host, may be NULL: nonzero asks for 16-bit
 *                             coordinates for the path; granted when every
 *                             coordinate of the path is an integer in
 *                             [-32768, 32767], else the path stays 32-bit
 * (Transforms do not change the sizes.)
 * Outputs (host): n_tags and n_words (32-bit words of the path data stream).
 * Segments whose control points all equal the current point are dropped; a
 * closed subpath -- every subpath of a fill -- whose end differs from its start
 * gets a closing line; every drawn subpath ends with a cap-marker tag; a path
 * with nothing to draw gets one empty tag.
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_INVALID_INPUT. */
se_status se_encode_size(const uint8_t* verbs, uint64_t n_verbs, const float* pts, uint64_t n_pts,
                         const uint32_t* path_verb_off, uint32_t n_paths, const se_style* styles,
                         const uint8_t* coord16, uint64_t* n_tags, uint64_t* n_words);

/* Encode a verb scene (all pointers host).  styles_in[n_paths] is the style of
 * each path; tags_out[n_tags], words_out[n_words] and styles_out[n_paths] must
 * be sized from se_encode_size (with the same coord16).  Consecutive paths with identical styles
 * share one style entry; *n_styles_out receives the number of entries.
 * transforms_in[6 * n_paths] (may be NULL: every path untransformed) gives each
 * path's affine transform (a b c d e f: x' = a x + c y + e, y' = b x + d y + f,
 * Section 8.2); consecutive paths with identical transforms share one entry of
 * transforms_out[6 * n_paths] (required when transforms_in is given), and
 * *n_transforms_out (may be NULL) receives the number of entries (0 without
 * transforms_in).  The expansion strokes the transformed path with half-width
 * h sqrt|ad - bc|; dash lengths are measured before the transform.
 * Coordinates and transforms must be finite; for a stroke half_width finite and
 * > 0 and miter_limit >= 1 (a fill's stroke fields are not checked).
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_INVALID_INPUT. */
se_status se_encode(const uint8_t* verbs, uint64_t n_verbs, const float* pts, uint64_t n_pts,
                    const uint32_t* path_verb_off, uint32_t n_paths, const se_style* styles_in,
                    const float* transforms_in, const uint8_t* coord16, uint8_t* tags_out, uint32_t* words_out,
                    se_style* styles_out, uint32_t* n_styles_out, float* transforms_out,
                    uint32_t* n_transforms_out);

/* ------------------------------------------------------------------------ */
/* Device expansion                                                          */
/* ------------------------------------------------------------------------ */
typedef struct se_ctx se_ctx;

/* The caller's device allocator.  alloc returns `bytes` of device memory on the
 * context's device that may be used in stream order on `cuda_stream` (the
 * stream the library will use it on), or NULL when it cannot; free gives back
 * a block alloc returned, once the library has enqueued its last use of it on
 * `cuda_stream` (stream-ordered release, as cudaFreeAsync).  `user` is passed
 * through unchanged.  Both are called from the thread that makes the library
 * call (for a server: from its worker threads) and never while a stream
 * capture is in progress.  A PyTorch caller passes its caching allocator, so
 * the library's workspace comes from the same pool as the tensors around it. */
typedef void* (*se_alloc_fn)(size_t bytes, void* user, void* cuda_stream);
typedef void (*se_free_fn)(void* ptr, void* user, void* cuda_stream);

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns a
 * growable device workspace (per-tag scan results, counts, offsets, status),
 * and every device buffer the library allocates for it (workspace, dash
 * workspace, host-path buffers, batch tables, library-owned scenes and
 * outlines, coverage scratch) comes from alloc_fn / free_fn.  Pass both NULL
 * for the CUDA stream-ordered allocator (cudaMallocAsync / cudaFreeAsync);
 * passing one without the other is an invalid argument.  An allocation the
 * callback refuses (NULL) fails the call that needed it with SE_ERR_OOM and
 * leaves the context usable.
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_CUDA, SE_ERR_OOM. */
se_status se_ctx_create(int device, void* cuda_stream, se_alloc_fn alloc_fn, se_free_fn free_fn, void* user,
                        se_ctx** out);
se_status se_ctx_destroy(se_ctx* ctx);
/* Last error message of the context (never NULL; owned by the context). */
const char* se_ctx_last_error(const se_ctx* ctx);

/* An encoded scene in DEVICE memory (caller-owned, read-only for the call).
 * tags[n_tags] 16-byte aligned; words[n_words], the path data stream, 4-byte
 * aligned (may be NULL when n_words == 0: a scene of empty paths); styles[n_styles];
 * dashes[n_dashes] (may be NULL when no style dashes). */
typedef struct se_scene_dev {
    const uint8_t* tags;
    uint64_t n_tags;
    const uint32_t* words;
    uint64_t n_words;
    const se_style* styles;
    uint32_t n_styles;
    uint32_t n_paths;      /* number of PATH bits in tags */
    const float* dashes;
    uint32_t n_dashes;
    const float* transforms;  /* 6 floats per entry (a b c d e f); may be NULL when n_transforms == 0 */
    uint32_t n_transforms;    /* entries; a TRANSFORM bit past the last entry is a malformed tag */
} se_scene_dev;

/* Outline buffers in DEVICE memory (caller-owned).
 *   prims      capacity x 4 floats (x0 y0 x1 y1), 16-byte aligned
 *   curvature  capacity floats: signed curvature of each arc (arcs only; may be NULL for lines)
 *   path_id    capacity u32: path of each primitive (may be NULL)
 *   tag_offset n_tags + 1 u64: first primitive of each tag (may be NULL).  For a
 *              scene with dash patterns the tags are those of the dashed
 *              rewrite: n_tags is se_stats.n_tags after se_count of the scene
 *   path_offset n_paths + 1 u64: first primitive of each path (may be NULL)
 * Primitives are written in a deterministic order: tag by tag, and within a
 * segment's tag its Euler-spiral pieces (side +h, then side -h) followed by
 * its join or end cap; a cap-marker tag holds its subpath's start cap.  A
 * dashed subpath contributes, per dash in order, one tag per source-segment
 * part the dash covers and a cap marker; a path left with no dash keeps one
 * empty tag. */
typedef struct se_outline_dev {
    float* prims;
    float* curvature;
    uint32_t* path_id;
    uint64_t* tag_offset;
    uint64_t* path_offset;
    uint64_t capacity;
} se_outline_dev;

/* Expand a device scene into the outline buffers, enqueued on the context
 * stream without any host synchronisation: [dash pass,] tag scan, plan
 * (subdivision), pieces, primitive scan, emit.  The dash pass runs when the
 * scene has a dash array (n_dashes > 0); styles with dash_count == 0 stay
 * solid.  If the total exceeds out->capacity nothing is written and se_sync
 * reports SE_ERR_CAPACITY; if the scene has more Euler-spiral pieces (or, when
 * dashed, more dash output) than the context's workspace holds, se_sync
 * reports SE_ERR_WORKSPACE (run se_count on the scene once: it sizes the
 * workspace).  A dash pattern with a negative or non-finite entry or offset,
 * or one that puts more than 2^23 periods on one subpath or 2^22 boundaries on
 * one segment, makes se_sync report SE_ERR_INVALID_INPUT; a pattern whose
 * entries sum to zero draws nothing.
 * The scene and outline buffers must stay alive until the work completes.
 * Errors at enqueue time: SE_ERR_INVALID_ARG, SE_ERR_OOM (workspace), SE_ERR_CUDA. */
se_status se_expand(se_ctx* ctx, const se_scene_dev* scene, const se_params* params, const se_outline_dev* out);

/* Count only: every stage but the emit, then wait for the stream and return
 * the number of primitives the scene expands to (host).  Grows the context's
 * workspace to fit the scene.  A following se_expand of the same scene with
 * the same params produces exactly that many primitives. */
se_status se_count(se_ctx* ctx, const se_scene_dev* scene, const se_params* params, uint64_t* n_prims);

/* The expansion that follows se_count of the same scene with the same params:
 * the count already left the scene's subdivision, pieces and offsets in the
 * context's workspace, so only the primitive scan (now writing the outline's
 * tag and path offsets) and the emit run -- the dash pass, tag scan, plan and
 * piece passes are not repeated.  The result is the one se_expand gives.
 * Enqueued on the context stream without host synchronisation.  Valid only as
 * the next expansion call on the context after that se_count (any other
 * count or expansion in between, or a different scene or params, gives
 * SE_ERR_INVALID_ARG); it can be issued once per count.
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_CUDA. */
se_status se_expand_counted(se_ctx* ctx, const se_scene_dev* scene, const se_params* params,
                            const se_outline_dev* out);

/* Wait for the context stream and read back the result of the last
 * se_expand: *n_prims (may be NULL) receives its primitive count and the
 * return value is its device status (SE_OK, SE_ERR_CAPACITY, SE_ERR_WORKSPACE,
 * SE_ERR_LIMIT, SE_ERR_INVALID_INPUT, SE_ERR_TIMEOUT) or SE_ERR_CUDA. */
se_status se_sync(se_ctx* ctx, uint64_t* n_prims);

/* Device address of the context's u64 primitive total of the last expansion
 * (valid until the next call on the context); lets a caller read it from a
 * stream without a host round trip. */
se_status se_total_device(se_ctx* ctx, const uint64_t** d_total);

/* End-to-end convenience on HOST buffers: upload the encoded streams (host
 * pointers), expand, and copy the primitives back into host_prims
 * (capacity x 4 floats) and host_curvature (capacity floats, arcs; may be
 * NULL).  Blocks until done; *n_prims receives the count.  Returns
 * SE_ERR_CAPACITY (with *n_prims set) when capacity is too small.  For large
 * scenes the emit runs in tag ranges and each range's block of the outline is
 * copied to the host on a second stream while the next range is emitted. */
se_status se_expand_host(se_ctx* ctx, const uint8_t* tags, uint64_t n_tags, const uint32_t* words,
                         uint64_t n_words, const se_style* styles, uint32_t n_styles, uint32_t n_paths,
                         const float* dashes, uint32_t n_dashes, const float* transforms, uint32_t n_transforms,
                         const se_params* params,
                         float* host_prims, float* host_curvature, uint64_t capacity, uint64_t* n_prims);

/* Sizes of the last expansion (waits for the stream).  Measurement support:
 * lets a caller account for the bytes each stage moves. */
typedef struct se_stats {
    uint64_t n_tags;         /* tags the last expansion ran over (after the dash rewrite, if any) */
    uint64_t n_input_tags;   /* tags of the last scene as given */
    uint64_t n_items;        /* Euler-spiral pieces + one join/cap item per tag */
    uint64_t n_prims;        /* output primitives */
    uint32_t piece_bytes;    /* size of one piece record */
    uint32_t tail_bytes;     /* size of one join/cap record */
    uint64_t workspace_bytes;
} se_stats;
se_status se_ctx_stats(se_ctx* ctx, se_stats* out);

/* Stage timing (not part of the paper's method: measurement support).
 * When enabled, se_expand records CUDA events on the context stream between
 * its stages.  se_profile_read waits for the stream and returns the stage
 * durations in milliseconds (ms[6]): ms[0] tag scan, ms[1] plan (subdivision),
 * ms[2] pieces (item scan, decode, piece setup), ms[3] primitive scan,
 * ms[4] emit, ms[5] dash pass (0 for a scene without dashes).
 * Errors: SE_ERR_INVALID_ARG (no profiled expansion yet), SE_ERR_CUDA. */
se_status se_profile_enable(se_ctx* ctx, int enable);
se_status se_profile_read(se_ctx* ctx, float* ms);

/* ------------------------------------------------------------------------ */
/* Library-owned scenes and outlines (the object form of the boundary)       */
/* ------------------------------------------------------------------------ */
/* A scene is built path by path with the SVG-style verbs of Section 8.1, or
 * made from already encoded streams (Table 1); se_scene_upload encodes a built
 * scene on the host (Section 8.2) and copies it to the context's device
 * (asynchronously on the context stream).  se_scene_expand counts the scene,
 * which waits for the stream, allocates a library-owned outline of exactly
 * that size and enqueues the expansion (tolerance split fit 0.2 / flatten 1.0);
 * se_outline_sync waits for it.  An outline still in flight is synchronised
 * by the next expansion its context starts (the context's count and status
 * read-back is its own until then).  The library owns scenes and outlines
 * until their _destroy; an outline keeps its device memory alive by itself.
 * Destroy scenes and outlines before their context, and keep a scene handed
 * to se_server_submit_scene alive until its request is released.
 * Errors: SE_ERR_INVALID_ARG (NULL, a builder call out of order, a scene of
 * another context), SE_ERR_INVALID_INPUT (non-finite coordinates, a bad dash
 * length, a path not starting with move_to), SE_ERR_OOM, SE_ERR_CUDA, and the
 * expansion's own codes from se_outline_sync. */
typedef struct se_scene se_scene;
typedef struct se_outline se_outline;

se_status se_scene_begin(se_ctx* ctx, se_scene** out);
/* open a path with its style (copied); the style's dash_first indexes the
 * scene's own dash lengths (se_dash_pattern) */
se_status se_path_begin(se_scene* scene, const se_style* style);
se_status se_move_to(se_scene* scene, float x, float y);
se_status se_line_to(se_scene* scene, float x, float y);
se_status se_cubic_to(se_scene* scene, float x1, float y1, float x2, float y2, float x3, float y3);
se_status se_close(se_scene* scene);
se_status se_path_end(se_scene* scene);
/* ask for 16-bit coordinates for the paths begun after this call (granted per
 * path when all its coordinates are integers in the 16-bit range) */
se_status se_set_coord16(se_scene* scene, int enable);
/* a quadratic Bezier segment (SE_VERB_QUAD) */
se_status se_quad_to(se_scene* scene, float x1, float y1, float x2, float y2);
/* the affine transform (6 floats a b c d e f; NULL = identity) of the paths begun
 * after this call (Section 8.2) */
se_status se_set_transform(se_scene* scene, const float* m);
/* append n dash lengths to the scene; *first_out receives their first index */
se_status se_dash_pattern(se_scene* scene, const float* lens, uint32_t n, uint32_t* first_out);
/* a scene from encoded HOST streams (copied): tags[n_tags], words[n_words],
 * styles[n_styles], n_paths PATH bits, dashes[n_dash] (may be NULL when 0),
 * transforms[6 * n_transforms] (may be NULL when 0) */
se_status se_scene_from_streams(se_ctx* ctx, const uint8_t* tags, size_t n_tags, const uint32_t* words, size_t n_words,
                                const se_style* styles, size_t n_styles, uint32_t n_paths, const float* dashes,
                                size_t n_dash, const float* transforms, size_t n_transforms, se_scene** out);
se_status se_scene_upload(se_scene* scene);
/* the uploaded scene's device descriptor (pointers owned by the scene) */
se_status se_scene_device(const se_scene* scene, se_scene_dev* out);
se_status se_scene_destroy(se_scene* scene);

/* Count (waits for the stream), allocate and enqueue the expansion of a scene
 * (uploaded first if it is not yet) at tolerance tol into a new outline. */
se_status se_scene_expand(se_scene* scene, float tol, uint32_t out_kind, se_outline** out);
/* Expand n scenes as one batch (se_batch_*); outs[d] receives scene d's
 * outline (the outlines share one buffer).  Waits for the expansion. */
se_status se_expand_batch(se_ctx* ctx, se_scene* const* scenes, uint32_t n, float tol, uint32_t out_kind,
                          se_outline** outs);
/* Wait for the outline; *n_prims and *n_paths (either may be NULL) receive its
 * sizes; returns the expansion's status. */
se_status se_outline_sync(se_outline* outline, uint64_t* n_prims, uint32_t* n_paths);
/* Device pointers of a synchronised outline: prims (n_prims x 4 floats),
 * curvature (arcs, else NULL) and path_offset (n_paths + 1 entries, relative
 * to the whole buffer: subtract path_offset[0] for this outline's own) */
se_status se_outline_device(const se_outline* outline, const float** prims, const float** curvature,
                            const uint64_t** path_offset);
/* Copy a synchronised outline into caller HOST buffers (any may be NULL):
 * prims n_prims x 4, curvature n_prims, path_offset n_paths + 1 (from 0). */
se_status se_outline_copy(const se_outline* outline, float* host_prims, float* host_curvature,
                          uint64_t* host_path_offset);
se_status se_outline_destroy(se_outline* outline);

/* ------------------------------------------------------------------------ */
/* Nonzero coverage of an outline (the downstream use of the line soup)      */
/* ------------------------------------------------------------------------ */
/* Section 8.1's renderer bins the line soup into tiles and computes pixel
 * coverage with scanlines; this entry point does that for a check and for
 * consumers of the outline.  For a W x H grid of pixel centres (x + 1/2,
 * y + 1/2) and every path, the winding number of the path's primitives
 * (crossings of the centre's row, counted with their direction); a pixel is
 * covered by a path when it is nonzero.  All pointers DEVICE:
 *   prims      n_prims x 4 floats (x0 y0 x1 y1), 16-byte aligned
 *   curvature  n_prims floats (arcs: signed curvature, > 0 turning left), or
 *              NULL for lines; arcs are cut into chords of sagitta <= 1e-3
 *   path_id    n_prims u32 (< n_paths)
 *   count      width * height u32, row-major: paths covering each pixel
 *   path_area  n_paths u64 (may be NULL): pixels each path covers
 * Blocks until done (the bucket and crossing counts size its temporaries).
 * Errors: SE_ERR_INVALID_ARG (also a grid of 2^40 pixels or more, or of 2^31
 * rows or columns or more, 2^32 or more (path, row) pairs with crossings, or 2^31 or more
 * crossings in all), SE_ERR_INVALID_INPUT (a path id out of range), SE_ERR_OOM,
 * SE_ERR_TIMEOUT, SE_ERR_CUDA. */
se_status se_coverage(se_ctx* ctx, const float* prims, const float* curvature, const uint32_t* path_id,
                      uint64_t n_prims, uint32_t n_paths, uint32_t width, uint32_t height, uint32_t* count,
                      uint64_t* path_area);

/* ------------------------------------------------------------------------ */
/* Batched expansion (many documents, one launch sequence, one CUDA graph)   */
/* ------------------------------------------------------------------------ */
/* Not part of the paper's method, which expands one scene per dispatch: a
 * batch serves many independent documents with one launch sequence.  The
 * documents are gathered into one scene (one kernel); each document's
 * primitives are then the contiguous range of the outline between the path
 * offsets of its first path and of the next document's first path, and are
 * identical to those of se_expand on the document alone. */
typedef struct se_batch se_batch;

/* Build a batch of n_docs device scenes (docs is a HOST array of descriptors
 * whose pointers are device pointers; the documents must stay alive and keep
 * their sizes while the batch exists; their contents are gathered each time
 * the batch is counted, expanded or its graph is launched, so a document may
 * be updated in place between launches).  Allocates the batch scene on the
 * context's device and waits for the context stream.
 * Errors: SE_ERR_INVALID_ARG (NULL pointers, or more than 2^31 tags / 2^32
 * points in total), SE_ERR_OOM, SE_ERR_CUDA. */
se_status se_batch_create(se_ctx* ctx, const se_scene_dev* docs, uint32_t n_docs, se_batch** out);
se_status se_batch_destroy(se_batch* batch);

/* First path of each document in the batch (host array of n_docs + 1; the
 * last entry is the total): document d owns outline paths
 * [path_first[d], path_first[d + 1]). */
se_status se_batch_doc_paths(const se_batch* batch, uint64_t* path_first);

/* The gathered scene (device pointers owned by the batch), e.g. for sizing
 * tag_offset; its contents are valid after a count, expand or launch. */
se_status se_batch_scene(const se_batch* batch, se_scene_dev* scene);

/* Gather, then se_count / se_expand the batch scene (same semantics). */
se_status se_batch_count(se_batch* batch, const se_params* params, uint64_t* n_prims);
se_status se_batch_expand(se_batch* batch, const se_params* params, const se_outline_dev* out);
/* se_expand_counted of the batch scene after se_batch_count (no second gather). */
se_status se_batch_expand_counted(se_batch* batch, const se_params* params, const se_outline_dev* out);

/* Capture gather + expansion into a CUDA graph (replacing an earlier
 * capture).  Run se_batch_count with the same params first: a capture never
 * allocates, and fails with SE_ERR_WORKSPACE if the workspace is too small.
 * Waits for the context stream; captures on a stream of the batch's own. */
se_status se_batch_capture(se_batch* batch, const se_params* params, const se_outline_dev* out);
/* Launch the captured graph on the context stream (asynchronous; se_sync
 * reads the result).  The graph holds the addresses of the context's
 * workspace: once the workspace has been reallocated (a count or expansion of
 * a larger scene on the same context), capture again.
 * Errors: SE_ERR_INVALID_ARG (nothing captured, or the workspace was
 * reallocated since the capture), SE_ERR_CUDA. */
se_status se_batch_launch(se_batch* batch);

/* ------------------------------------------------------------------------ */
/* Launch tuning                                                             */
/* ------------------------------------------------------------------------ */
/* Launch shapes of the expansion kernels; the output does not depend on them. */
typedef struct se_tuning {
    uint32_t plan_block;          /* threads per block of the per-tag kernels: 64, 128 or 256 */
    uint32_t piece_block;         /* the per-piece pass's tile: records staged in shared memory per
                                     block, 128 or 256 (64 is taken as 128) */
    uint32_t emit_block;          /* threads per block of the emit kernels: 64 or 128 */
    uint32_t emit_blocks_per_sm;  /* resident emit blocks per SM, 1..32 (0: as many as fit) */
} se_tuning;
se_status se_get_tuning(const se_ctx* ctx, se_tuning* tuning);
/* Errors: SE_ERR_INVALID_ARG (a value out of range). */
se_status se_set_tuning(se_ctx* ctx, const se_tuning* tuning);
/* Time `reps` expansions of the scene into `out` under candidate tunings
 * (coordinate descent over emit_block, emit_blocks_per_sm, plan_block and the
 * piece tile), keep the fastest on the context
 * and return it in *chosen (may be NULL).  Run se_count on the scene first.
 * Synchronous; leaves the last expansion's result in `out`. */
se_status se_autotune(se_ctx* ctx, const se_scene_dev* scene, const se_params* params, const se_outline_dev* out,
                      int reps, se_tuning* chosen);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching under an HBM budget                          */
/* ------------------------------------------------------------------------ */
/* Not part of the paper's method: a runtime that serves expansion requests
 * as they arrive.  Each slot (a worker thread with its own context, CUDA
 * stream and workspace) takes the queued requests that share the oldest
 * request's parameters, up to max_batch_docs documents and max_batch_tags
 * tags, counts them as one batch (se_batch_*), waits until the batch's
 * gathered encodings and outline fit in the HBM budget next to everything
 * in flight or held, expands it and hands each request its range of the batch
 * outline.  Requests arriving meanwhile go to the next free slot, so batches
 * overlap on the device.  A batch too large for the budget is split; a single
 * request too large fails with SE_ERR_BUDGET.  Results are bit-identical to
 * expanding each document alone. */
typedef struct se_server se_server;

typedef struct se_server_config {
    uint32_t slots;           /* concurrent batches, 1..64 */
    uint32_t max_batch_docs;  /* documents per batch, >= 1 (1: one expansion per document) */
    uint64_t max_batch_tags;  /* no further document joins a batch past this many tags (0: no limit) */
    uint64_t hbm_budget;      /* bytes of gathered encodings + outline buffers in flight or held */
    se_alloc_fn alloc_fn;     /* device allocator of every slot's context and of the outlines (both */
    se_free_fn free_fn;       /*   NULL: the CUDA stream-ordered allocator); see se_ctx_create */
    void* alloc_user;
} se_server_config;

typedef struct se_request_result {
    int32_t done;             /* 0 while queued or running */
    int32_t status;           /* when done: SE_OK, SE_ERR_LIMIT, SE_ERR_BUDGET or the expansion's error */
    uint32_t batch_docs;      /* documents in the batch the request ran in */
    uint32_t reserved;
    const float* prims;       /* device: n_prims x 4 floats (x0 y0 x1 y1), valid until released */
    const float* curvature;   /* device: n_prims floats for arc output, else NULL */
    uint64_t n_prims;
    int64_t t_submit_ns, t_start_ns, t_done_ns;  /* steady clock, since the server was created */
} se_request_result;

typedef struct se_server_stats {
    uint64_t submitted, completed, failed, batches, queued;
    uint32_t max_concurrent;  /* most batches that ran at once */
    uint32_t reserved;
    uint64_t bytes_in_use, bytes_peak, hbm_budget;
} se_server_stats;

/* Start a server on CUDA device `device` (threads and streams of its own).
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_CUDA, SE_ERR_OOM. */
se_status se_server_create(int device, const se_server_config* config, se_server** out);
/* Stop the workers (a running batch finishes; queued requests are dropped)
 * and free every held outline. */
se_status se_server_destroy(se_server* server);
/* Queue a request: `doc` points to a device scene that must stay alive and
 * unchanged until the request is done.  Thread-safe; returns at once. */
se_status se_server_submit(se_server* server, const se_scene_dev* doc, const se_params* params, uint64_t* req_id);
/* State of a request (wait != 0: block until it is done). */
se_status se_server_poll(se_server* server, uint64_t req_id, int wait, se_request_result* out);
/* Give back a done request's outline memory (and forget the request). */
se_status se_server_release(se_server* server, uint64_t req_id);
se_status se_server_get_stats(se_server* server, se_server_stats* out);
/* The cause of the server's most recent failed batch (the step and the library's or
 * CUDA's message; "" when none failed), copied into buf: len bytes, NUL-terminated,
 * truncated to fit.  Errors: SE_ERR_INVALID_ARG (NULL server or buf, len 0). */
se_status se_server_last_error(se_server* server, char* buf, size_t len);
/* Queue a request for a library-owned scene (uploaded and synchronised first;
 * it must stay alive until the request is done). */
se_status se_server_submit_scene(se_server* server, se_scene* scene, float tol, uint32_t out_kind, uint64_t* req_id);

/* ------------------------------------------------------------------------ */
/* Offsets without allocation                                               */
/* ------------------------------------------------------------------------ */

/* Test hook for the bounded waits (the paper has no counterpart).  Runs the
 * library's look-back scan over n counts (in scratch from the context's
 * allocator) with the first tile's ticket never handed out, so the first tile
 * never publishes its prefix -- a flag that nothing sets -- and the second
 * tile's wait on it gives up after spin_limit polls.  The kernel then records
 * SE_ERR_TIMEOUT in its status word and returns; nothing faults or hangs, and
 * the context stays usable.  Every expansion kernel that indexes by a scan's
 * offsets skips its writes once a wait has given up.
 * n > 4096 (two scan tiles or more), n < 2^32, spin_limit >= 1.  Synchronises
 * the context's stream.  Returns SE_ERR_TIMEOUT when the wait ran out (the
 * expected outcome), SE_OK if it did not.
 * Errors: SE_ERR_INVALID_ARG, SE_ERR_OOM, SE_ERR_CUDA. */
se_status se_debug_scan_timeout(se_ctx* ctx, uint64_t n, uint32_t spin_limit);

/* Test hook for the emit kernels' bulk copies (one-dimensional copies from
 * global to shared memory on the copy engine, completed through a shared-memory
 * barrier; the paper has no counterpart).  One warp waits on a fresh barrier's
 * first phase, polling at most spin_limit times.  copy = 0: nothing is issued,
 * so the wait runs out (a phase that nothing completes), the kernel records
 * SE_ERR_TIMEOUT and returns; nothing faults or hangs and the context stays
 * usable.  copy != 0: 256 bytes are copied first and checked; the wait succeeds
 * unless spin_limit is too short for the copy to land (the kernel then lets the
 * copy drain before it exits).  Scratch comes from the context's allocator;
 * synchronises the context's stream.  Returns SE_ERR_TIMEOUT when the wait ran
 * out, SE_OK when the copy landed intact.
 * Errors: SE_ERR_INVALID_ARG (spin_limit 0), SE_ERR_OOM, SE_ERR_CUDA (including
 * wrong bytes delivered). */
se_status se_debug_bulk_timeout(se_ctx* ctx, uint32_t spin_limit, int copy);

/* Largest number of counts se_scan_offsets_noalloc accepts (2^24). */
#define SE_NOALLOC_MAX_COUNTS (1ull << 24)

/* Exclusive scan of counts[0..n) (u32, device) into offsets[0..n] (u64,
 * device; offsets[n] = the total): the count -> offset step of the expansion,
 * for callers that may not allocate device memory -- code under a device
 * memory budget reserved up front, a render loop that must not block on the
 * allocator, a plugin whose host application owns every device allocation.
 * The paper has no counterpart: its shader reserves output by atomic bump
 * allocation.
 *
 * It allocates nothing: its scratch (look-back state for up to
 * SE_NOALLOC_MAX_COUNTS counts, about 80 KB) is a fixed array in the library
 * that every GPU loading the library holds until the process exits.  The
 * first call on a device resolves that array's device address (with the
 * device current).  Every call shares the one array and clears its state at
 * the start, so calls that overlap on the GPU (other streams, other threads)
 * race: serialise them.  Runs on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream), reads the scan's status word back on that stream and waits
 * for that stream alone before returning.  Because it waits on the stream,
 * the call cannot be recorded into a CUDA graph by stream capture.
 * Errors: SE_ERR_INVALID_ARG (NULL pointer, or n > SE_NOALLOC_MAX_COUNTS),
 * SE_ERR_TIMEOUT (a bounded wait of the scan gave up), SE_ERR_CUDA. */
se_status se_scan_offsets_noalloc(const uint32_t* counts, uint64_t n, uint64_t* offsets, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* STROKE_EXPAND_H */
