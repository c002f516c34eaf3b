/*
 * gpphot.h -- C ABI of the GB300 (sm_103a) per-frame source-extraction path.
 *
 * The operations follow the GPU stages of the GPUPHOT paper (arXiv
 * 2609.32375): a local background with a per-pixel noise map (Section 3.1),
 * matched-filter detection against a significance threshold with
 * first-moment centroids (Section 3.2) and circular-aperture sums accumulated
 * at float64 accuracy with propagated variance (Section 3.4).  Where the
 * paper leaves the algorithm open the library implements the SExtractor-style
 * reading: sigma-clipped mesh statistics, natural-spline maps, labelled
 * segments with moments and exact disc/pixel overlap apertures.
 *
 * Conventions (every entry point):
 *  - All array pointers are DEVICE pointers owned by the caller unless the
 *    comment says "host".  Images are row-major, x = column, y = row,
 *    pixel (x, y) covers [x-1/2, x+1/2] x [y-1/2, y+1/2], linear index
 *    L = y * width + x.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns without waiting.  Outputs are valid once the stream
 *    has synchronised.  Arguments are checked on the host before any launch;
 *    an argument error returns GP_ERR_INVALID_ARG with nothing enqueued.
 *  - Conditions only the device can see (catalog capacity exceeded, an
 *    internal table full, a bounded wait that gave up) are recorded in the
 *    context's device status word; gp_ctx_sync() returns it.
 *  - Scratch memory comes only from the context's workspace arena, which is
 *    allocated once by gp_ctx_create(); no entry point allocates.  Calls on
 *    one context share that arena, so calls on one context must be ordered
 *    (same stream, or synchronised) -- use one context per concurrent stream.
 *  - There is no CPU fallback: without a usable sm_103a device the calls
 *    fail with GP_ERR_CUDA.
 */
#ifndef GPPHOT_H
#define GPPHOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gp_stream; /* a cudaStream_t */

typedef enum {
    GP_OK = 0,
    GP_ERR_INVALID_ARG = 1,     /* rejected on the host, nothing enqueued */
    GP_ERR_OOM = 2,             /* workspace arena too small (or allocation failed in create) */
    GP_ERR_CAPACITY = 3,        /* more sources than catalog rows (device-side) */
    GP_ERR_CUDA = 4,            /* a CUDA runtime call failed */
    GP_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up */
    GP_ERR_NOT_IMPLEMENTED = 6,
    GP_ERR_INTERNAL = 7         /* an internal device table overflowed */
} gp_status;

typedef enum { GP_U16 = 0, GP_F32 = 1 } gp_dtype;

/* per-source / per-aperture flag bits */
enum {
    GP_FLAG_SAT = 1u,                 /* a pixel >= saturation in the segment / under the disc */
    GP_FLAG_CENTROID_FALLBACK = 2u,   /* segment sum <= 0: unweighted centroid and moments */
    GP_FLAG_TRUNCATED = 4u,           /* aperture disc extends beyond the frame */
    GP_FLAG_BAD = 8u                  /* aperture disc covers a masked / NaN pixel */
};

typedef struct gp_ctx gp_ctx;

/* Create a context on `device` with a workspace arena of `workspace_bytes`
 * (0: 2 GiB).  gp_workspace_bytes() gives the size one frame needs.
 * Returns GP_ERR_OOM if the arena cannot be allocated. */
gp_status gp_ctx_create(int device, size_t workspace_bytes, gp_ctx** out);
void gp_ctx_destroy(gp_ctx* ctx);

/* Message for the last non-OK status returned on this host thread. */
const char* gp_last_error(void);

/* Synchronise `stream` and return the device-side status of the work enqueued
 * on this context since the previous gp_ctx_sync (then reset it to GP_OK). */
gp_status gp_ctx_sync(gp_ctx* ctx, gp_stream stream);

/* Stage timing.  When enabled, every call records CUDA events on its stream
 * at the boundaries of its stages (box statistics; mesh filter and spline
 * tables; threshold pass; tile labelling; tile merge; label ranking;
 * moments and apertures) into a ring of 256 call slots.  gp_ctx_stats() waits for the
 * recorded events, returns the device time of each stage summed over the
 * calls recorded since the previous gp_ctx_stats() (at most the last 256),
 * and starts a new accumulation.  Disabled by default; the events add a few
 * microseconds per call. */
#define GP_NSTAGES 7
typedef struct {
    int32_t calls;                 /* calls summed */
    int32_t launches;              /* kernels launched by the most recent call */
    float ms[GP_NSTAGES];          /* summed device milliseconds per stage */
} gp_stats;
gp_status gp_ctx_set_timing(gp_ctx* ctx, int32_t enable);
gp_status gp_ctx_stats(gp_ctx* ctx, gp_stats* out);

/* Failure detection.  The tile merge of segments across detection tiles
 * (Section 3.2's segmentation, kept exact across tiles) walks union-find
 * chains in device memory; every walk is bounded.  A walk that runs out of
 * steps stops, records GP_ERR_TIMEOUT in the context's device status word
 * (returned by the next gp_ctx_sync) and leaves that frame's segments
 * incomplete; the stream and the context stay usable.  `steps` sets the
 * bound for later calls on this context (0: the default, 2^22, far above
 * any chain a frame can build).  GP_ERR_INVALID_ARG for steps < 0. */
gp_status gp_ctx_set_walk_limit(gp_ctx* ctx, int32_t steps);

/* Arena bytes needed to run gp_extract on a width x height frame with this
 * mesh size and catalog capacity (capacity <= 0: the default internal table
 * size of max(65536, width*height/32) segments). */
size_t gp_workspace_bytes(int32_t width, int32_t height, int32_t mesh, int32_t capacity);

/* ---------------------------------------------------------------- inputs */
typedef struct {
    const void* data;      /* device; uint16 or float32 pixels */
    gp_dtype dtype;
    int32_t width, height;
    int64_t pitch;         /* elements between rows, >= width */
    const uint8_t* mask;   /* device width*height (pitch = width), nonzero = bad; nullable */
    float saturation;      /* pixels >= saturation are flagged; <= 0: none */
} gp_image;

/* Background parameters (Section 3.1): mesh box side, median filter size of
 * the box meshes, clip factor k and the maximum number of clip passes. */
typedef struct {
    int32_t mesh;          /* 16 .. 256 (uint16 frames); 16 .. 128 (float32 frames) */
    int32_t filter_size;   /* odd, 1 .. 7; 1 = no mesh filtering */
    float clip_k;          /* >= 1, typically 3 */
    int32_t clip_maxiter;  /* >= 0, typically 10 */
} gp_bkg_params;

/* Background result: the filtered box meshes (my rows of mx boxes), from
 * which the per-pixel background B(p) and noise sigma(p) are the
 * tensor-product natural cubic spline through the box centres. */
typedef struct {
    int32_t mesh;          /* box side used */
    int32_t mx, my;        /* mesh size: ceil(width/mesh), ceil(height/mesh) */
    float* bkg_mesh;       /* device my*mx, caller-owned */
    float* rms_mesh;       /* device my*mx, caller-owned */
    float* bkg_map;        /* device width*height full-resolution B(p); nullable (not written) */
    float* rms_map;        /* device width*height full-resolution sigma(p); nullable */
} gp_bkg;

/* Detection parameters (Section 3.2): the matched-filter kernel (host,
 * kh rows of kw taps, both odd <= 15; normalised to unit sum inside; a zero
 * sum is rejected), the threshold in units of sigma(p) and the minimum
 * segment area in pixels. */
typedef struct {
    const float* kernel;   /* HOST pointer, kh*kw taps */
    int32_t kw, kh;
    float thresh;          /* > 0 */
    int32_t minarea;       /* >= 1 */
    uint8_t* mask_out;     /* device width*height: the raw threshold mask (1 = foreground); nullable */
    int32_t* nnear;        /* device scalar: pixels with |F - k sigma| <= 1e-5 |k sigma|; nullable */
} gp_det_params;

/* Segment catalog, structure of arrays, `capacity` rows, ascending label.
 * label = 1 + minimum linear index of the segment; (x, y) is the first
 * moment of m = I - B over the segment; x2, y2, xy its central second
 * moments; peak is the maximum of m (position: its first pixel in raster
 * order). */
typedef struct {
    int32_t capacity;
    int32_t* n;            /* device scalar: number of segments found (may exceed capacity) */
    uint32_t* label;
    int32_t* npix;
    double* flux_iso;      /* sum of m over the segment */
    double *x, *y, *x2, *y2, *xy;
    int32_t *xmin, *xmax, *ymin, *ymax;
    float* peak;
    int32_t *xpeak, *ypeak;
    uint32_t* flags;
} gp_catalog;

/* Aperture parameters (Section 3.4): radii in pixels (host, nr <= 8) and the
 * gain for the Poisson term of the error (<= 0: no Poisson term). */
typedef struct {
    const float* radii;    /* HOST pointer */
    int32_t nr;
    float gain;
} gp_ap_params;

/* ------------------------------------------------------------ operations */

/* Section 3.1: per-box sigma-clipped statistics, invalid-box filling, mesh
 * median filter.  Fills bkg->bkg_mesh / rms_mesh (and the full maps when
 * their pointers are non-null).  bkg->mesh/mx/my are set by the call. */
gp_status gp_background(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* p,
                        gp_bkg* bkg, gp_stream stream);

/* Section 3.2: m = I - B, F = K (x) m (correlation, mirror border),
 * foreground F > thresh * sigma(p), 8-connected segments of at least
 * minarea pixels labelled 1 + min linear index (others 0) into `segmap`
 * (device width*height, caller-owned), and the segment catalog. */
gp_status gp_detect(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_det_params* p,
                    uint32_t* segmap, gp_catalog* cat, gp_stream stream);

/* Section 3.4: circular apertures of each radius around (x[i], y[i])
 * (device, n sources): flux = sum over in-frame good pixels of the exact
 * disc/pixel overlap area times m; fluxerr^2 = sum area * sigma(p)^2 +
 * max(flux, 0) / gain.  Outputs n*nr (source-major), device, caller-owned. */
gp_status gp_aperture(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg,
                      const double* x, const double* y, int32_t n, const gp_ap_params* p,
                      double* flux, double* fluxerr, uint32_t* flags, gp_stream stream);

/* Section 3.4, growth curves: for each source i and each integer radius
 * radii[k] (HOST array, nr of them, strictly increasing, 0 <= radius <=
 * GP_GROWTH_MAX_R, 1 <= nr <= GP_GROWTH_MAX_NR), the sum of m over the
 * top-hat {(u, v) : u^2 + v^2 <= radius^2} centred on the pixel nearest the
 * source, (floor(x[i] + 1/2), floor(y[i] + 1/2)): the value at that pixel of
 * the frame's cross-correlation with the top-hat, which the paper forms for
 * the whole frame by FFT.  Pixels outside the frame or bad (masked, NaN)
 * are left out and flagged GP_FLAG_TRUNCATED / GP_FLAG_BAD; GP_FLAG_SAT
 * marks a saturated pixel under the top-hat.  fluxerr^2 = sum of sigma(p)^2
 * over the same pixels + max(flux, 0) / gain (gain <= 0: no Poisson term).
 * x, y: device, n sources; flux, fluxerr, flags: device, n*nr
 * (source-major), caller-owned.  Sums are reproducible bit for bit.
 * GP_ERR_INVALID_ARG on a null array with n > 0, n < 0 or a radius list
 * outside the rules above; nothing is launched then. */
#define GP_GROWTH_MAX_NR 32
#define GP_GROWTH_MAX_R 255
gp_status gp_growth(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg,
                    const double* x, const double* y, int32_t n, const int32_t* radii,
                    int32_t nr, float gain, double* flux, double* fluxerr, uint32_t* flags,
                    gp_stream stream);

/* Section 3.4, optimal aperture radius.  The paper searches the radius of
 * largest S/N only on high-S/N isolated calibrators, fits
 * log10 r_opt = a log10 nu + b to them, with nu the detection significance,
 * and gives every other source the radius of the fit.  Here, for the
 * catalog rows min(*cat->n, cat->capacity) (device columns x, y, xpeak,
 * ypeak and flags as gp_extract leaves them):
 *  - the growth curves at the centroids, as gp_growth;
 *  - nu = F / sigma at the peak pixel, F the matched filter of gp_detect
 *    (dp's kernel; dp->thresh and dp->minarea are not used);
 *  - kopt, the radius index of largest S/N = flux / fluxerr (the first of
 *    equal values; S/N 0 where fluxerr <= 0);
 *  - calibrators: catalog flags 0, no growth flag at any radius, nu > 0,
 *    S/N at kopt >= snr_min, and no other row's centroid closer than d_iso;
 *  - the least-squares fit of log10 r[kopt] on log10 nu over the
 *    calibrators (fit = a, b, their number, status: 0 fitted, 1 fewer than
 *    three or all nu equal);
 *  - kfinal: a calibrator's kopt; for the others the grid radius nearest to
 *    10^(a log10 nu + b) (ties to the larger), or index 0 when nu <= 0 or
 *    the fit failed; flux_opt and fluxerr_opt are the growth curve there.
 * Every output is device memory, capacity rows (capacity*nr for the curves,
 * source-major; 4 doubles for fit), caller-owned.  GP_ERR_INVALID_ARG on a
 * null pointer, radii outside gp_growth's rules, snr_min not finite or
 * d_iso < 0; nothing is launched then. */
typedef struct {
    const int32_t* radii;  /* HOST pointer: the growth-curve radii */
    int32_t nr;
    float gain;            /* Poisson term of the errors (<= 0: none) */
    float snr_min;         /* calibrators: least S/N at their best radius */
    float d_iso;           /* calibrators: no other centroid closer (px) */
} gp_ropt_params;

typedef struct {
    double* flux;          /* capacity*nr growth curves */
    double* fluxerr;
    uint32_t* flags;
    float* nu;             /* capacity */
    int32_t* kopt;         /* capacity */
    uint8_t* calib;        /* capacity: 1 for a calibrator */
    int32_t* kfinal;       /* capacity */
    double* flux_opt;      /* capacity */
    double* fluxerr_opt;   /* capacity */
    double* fit;           /* 4 */
} gp_ropt_out;

gp_status gp_optimal_radius(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg,
                            const gp_det_params* dp, const gp_catalog* cat,
                            const gp_ropt_params* p, gp_ropt_out* out, gp_stream stream);

/* Section 3.2, the second detection pass with a spatially varying PSF: the
 * local PSF is a reference P0 plus K eigenmodes e_k weighted by coefficient
 * maps c_k, and the matched filter is the sum of K + 1 correlations,
 *   S(p) = (P0 (x) m)(p) + sum_k c_k(p) (e_k (x) m)(p),
 * with m = I - B (bad pixels 0) and a mirror border.  The kernels are used
 * as given (no normalisation).  c_k is the natural cubic spline through the
 * centres of square tiles of side `tile` holding the per-tile coefficients
 * (the background mesh's interpolation).  Foreground is S > thresh * sigma(p);
 * labelling, minarea, segmap and catalog are those of gp_detect. */
#define GP_PSF_MAX_MODES 8
typedef struct {
    const float* p0;       /* HOST: kh rows of kw taps */
    const float* modes;    /* HOST: K kernels of kh*kw taps, mode-major */
    int32_t K, kw, kh;     /* 0 <= K <= GP_PSF_MAX_MODES; kw, kh odd <= 15 */
    const float* coef;     /* DEVICE: K meshes of ceil(H/tile) rows of ceil(W/tile), mode-major */
    int32_t tile;          /* >= 1 */
    float thresh;          /* > 0 */
    int32_t minarea;       /* >= 1 */
} gp_psf_params;

/* segmap: device width*height, caller-owned; cat as in gp_detect.
 * GP_ERR_INVALID_ARG on a null pointer or a parameter outside the ranges
 * above; nothing is launched then. */
gp_status gp_detect_psf(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg,
                        const gp_psf_params* p, uint32_t* segmap, gp_catalog* cat,
                        gp_stream stream);

/* Section 3.1, the optional cosmetic corrections that precede the
 * background, each enabled by its parameters:
 *  - cosmic rays (cr_gain > 0), in the manner of L.A.Cosmic at the native
 *    scale: L = 4 I - (the four nearest neighbours), L+ = max(L, 0); the
 *    noise N = sqrt(max(med5(I), 0) cr_gain + cr_read_noise^2) / cr_gain
 *    (ADU; gain in e-/ADU, read noise in e-); S = L+ / (sqrt(20) N) less its
 *    5 x 5 median; the fine structure F = med3(I) - med7(med3(I)), at least
 *    0.01; a pixel is flagged where S > cr_sigclip and L+ / F > cr_objlim and
 *    takes the median of the good unflagged pixels of its 5 x 5 window;
 *  - then salt-and-pepper noise (rtn_t > 0): a pixel whose residual from its
 *    3 x 3 median exceeds rtn_t (ADU) in magnitude, with no such pixel among
 *    its 8 neighbours, takes the median.
 * Windows have a mirror border; bad pixels (the image's mask, non-finite
 * values) are left out of every window and are never flagged or changed.
 * out: device width*height float32, the corrected frame (bad pixels keep
 * their values).  flags (device width*height, nullable): bit 1 replaced by
 * the salt-and-pepper filter, bit 2 flagged as a cosmic ray.  counts
 * (device, 2 ints, nullable, cleared by the call): replaced, flagged.
 * GP_ERR_INVALID_ARG on a null out, both filters off, or cr_read_noise <= 0
 * with cr_gain > 0; GP_ERR_OOM when both are on and the workspace cannot hold
 * the intermediate frame (width*height floats). */
typedef struct {
    float rtn_t;
    float cr_gain, cr_read_noise, cr_sigclip, cr_objlim;
} gp_cosmetic_params;

gp_status gp_cosmetic(gp_ctx* ctx, const gp_image* img, const gp_cosmetic_params* p, float* out,
                      uint8_t* flags, int32_t* counts, gp_stream stream);

/* Multi-threshold deblending of the segments of `segmap` (the rows of `cat`,
 * as gp_detect or gp_extract leave them, with dp their detection kernel,
 * threshold and minarea).  The paper's detection takes local maxima and
 * does not deblend; this is the SExtractor reading.  For a segment of at
 * least 2 minarea pixels, nu = F / sigma: levels
 * t_i = thresh (nu_max / thresh)^(i / nthresh), i = 0..nthresh-1; the
 * branches of a level are the 8-connected components of {nu > t_i} in the
 * segment; a branch is significant with minarea pixels and a sum of m above
 * mincont times the segment's (which must be > 0); from the whole segment
 * upwards a branch hands on to its significant children, and one without is
 * a seed.  With two or more seeds the other pixels go to the seeds by growth
 * within the level sets from the highest level down (a pixel takes the
 * smallest rank, by first pixel, of its attributed 8-neighbours), and each
 * object is labelled 1 + its minimum linear index in `segmap` (in place).
 * `objects` receives a catalog row per object of the split segments, in
 * label order (the columns of gp_catalog; n = their number).  counts
 * (device, 2 ints, nullable): segments split, objects made.  The scratch is
 * the context's workspace; a segment that does not fit is left whole and
 * the call's status is GP_ERR_CAPACITY (as is more than 1024 objects in a
 * segment, or more objects than objects->capacity).  GP_ERR_INVALID_ARG on
 * null pointers, nthresh outside 1..64 or mincont outside [0, 1]. */
typedef struct {
    int32_t nthresh;       /* number of levels (SExtractor: 32) */
    float mincont;         /* minimum contrast (SExtractor: 0.005) */
} gp_deblend_params;

gp_status gp_deblend(gp_ctx* ctx, const gp_image* img, const gp_bkg* bkg, const gp_det_params* dp,
                     const gp_deblend_params* p, uint32_t* segmap, const gp_catalog* cat,
                     gp_catalog* objects, int32_t* counts, gp_stream stream);

/* The three stages in one call; apertures at each segment's centroid, rows
 * aligned with the catalog (capacity*nr). */
gp_status gp_extract(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* bp,
                     const gp_det_params* dp, const gp_ap_params* ap, gp_bkg* bkg,
                     uint32_t* segmap, gp_catalog* cat, double* flux, double* fluxerr,
                     uint32_t* apflags, gp_stream stream);

/* The labelling step of gp_detect alone on a caller-supplied mask (device
 * width*height, nonzero = foreground): same 8-connectivity, canonical labels
 * and minarea rule, so labels can be compared from an identical mask.
 * n_out (device scalar, nullable) receives the number of segments kept. */
gp_status gp_label_mask(gp_ctx* ctx, const uint8_t* mask, int32_t width, int32_t height,
                        int32_t minarea, uint32_t* segmap, int32_t* n_out, gp_stream stream);

/* ------------------------------------------------- learned background --
 * A small convolutional network maps one-pass per-box quantile features to
 * the background and rms meshes, in place of the iterative clip and median
 * filter.  The paper has no counterpart (its background is an FFT-smoothed
 * local estimate, Section 3.1); the plain estimator of gp_background stays
 * as the fallback and produces the training targets.
 *
 * Fixed architecture: six 3x3 convolutions, zero padding, ReLU between
 * layers, channels 5 -> 32 -> 48 -> 48 -> 32 -> 32 -> 2.  Activations are
 * NHWC bfloat16 (channels padded to 16, 32, 48, 48, 32, 32, 16); each layer's
 * weights are packed by gp_cnn_pack into bfloat16 [cout_p][9][cin_p] (tap =
 * 3 dy + dx, offsets -1..1) with float32 biases padded to cout_p. */
#define GP_CNN_LAYERS 6
typedef struct {
    const void* wt[GP_CNN_LAYERS];       /* device, packed bf16 forward weights */
    const float* bias[GP_CNN_LAYERS];    /* device, float32, cout_p entries */
} gp_cnn_weights;

/* The background stage with the network: per-box quantiles (one histogram
 * pass, no clipping), features, network, meshes, spline maps.  Same outputs
 * as gp_background (p->filter_size, clip_k and clip_maxiter are unused). */
gp_status gp_background_learned(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* p, const gp_cnn_weights* net,
                                gp_bkg* bkg, gp_stream stream);

/* gp_extract with the network's background (same arguments and outputs,
 * plus the weights). */
gp_status gp_extract_learned(gp_ctx* ctx, const gp_image* img, const gp_bkg_params* bp, const gp_det_params* dp,
                             const gp_ap_params* ap, const gp_cnn_weights* net, gp_bkg* bkg, uint32_t* segmap,
                             gp_catalog* cat, double* flux, double* fluxerr, uint32_t* apflags, gp_stream stream);

/* Per-box quantiles q10, q25, q50, q75, q90 of the good pixels (float32,
 * [5][my][mx], device, caller-owned), from one pass over the frame. */
gp_status gp_box_quantiles(gp_ctx* ctx, const gp_image* img, int32_t mesh, float* quant, gp_stream stream);

/* Network layers and training steps (all pointers device, caller-owned;
 * supported (cin_p, cout_p) pairs: (16,32) (32,48) (48,48) (48,32) (32,32)
 * (32,16)).  x, y: NHWC bf16 [n][h][w][c_p]; out_f32 writes float32
 * [n][h][w][creal] instead (the output layer). */
gp_status gp_cnn_conv3x3(const void* x, int32_t n, int32_t h, int32_t w, int32_t cin_p, const void* wt,
                         const float* bias, int32_t cout_p, int32_t relu, void* y, int32_t out_f32, int32_t creal,
                         gp_stream stream);
/* dW[cout][cin][3][3] and db[cout] from the layer input x and the gradient
 * dp at its pre-activation; partial (nslot*9*cout_p*cin_p floats) and bpart
 * (nslot*cout_p floats) are scratch; the slots are summed in a fixed order. */
gp_status gp_cnn_conv3x3_wgrad(const void* x, const void* dp, int32_t n, int32_t h, int32_t w, int32_t cin_p,
                               int32_t cout_p, int32_t cin, int32_t cout, int32_t nslot, float* partial, float* bpart,
                               float* dw, float* db, gp_stream stream);
/* dp = dy where y > 0, else 0 (bf16, count elements) */
gp_status gp_cnn_relu_backward(const void* dy, const void* y, void* dp, int64_t count, gp_stream stream);
/* mean squared error of pred vs target (float32 [npos][2]); writes
 * dL/dpred as bf16 [npos][cout_p] (zero in the padding) and *loss */
gp_status gp_cnn_mse(const float* pred, const float* target, int64_t npos, int32_t cout_p, void* dy, float* partial,
                     int32_t nblocks, float* loss, gp_stream stream);
/* master weights W[cout][cin][3][3] float32 and b[cout] -> forward weights
 * wt [cout_p][9][cin_p], data-gradient weights wtd [cin_p][9][cout_p]
 * (taps flipped), padded bias */
gp_status gp_cnn_pack(const float* W, const float* b, int32_t cin, int32_t cout, int32_t cin_p, int32_t cout_p,
                      void* wt, void* wtd, float* bias_p, gp_stream stream);
/* one AdamW step (decoupled weight decay, bias-corrected moments) */
gp_status gp_cnn_adamw(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                       float eps, float weight_decay, int32_t step, gp_stream stream);
/* features of nframes frames from their quantiles ([nframes][5][nbox]):
 * centre c = median box median, scale s = median (q75 - q25) / 1.349,
 * feat = (q - c) / s as bf16 [nframes][nbox][16]; norm = (c, s) per frame */
gp_status gp_cnn_features(const float* quant, int32_t nframes, int32_t nbox, void* feat, float* norm,
                          gp_stream stream);
/* plain meshes -> normalised training targets [nframes][nbox][2] */
gp_status gp_cnn_targets(const float* bkg_mesh, const float* rms_mesh, const float* norm, int32_t nbox,
                         int32_t nframes, float* target, gp_stream stream);
/* network output [nframes][nbox][2] -> meshes */
gp_status gp_cnn_denorm(const float* out, const float* norm, int32_t nbox, int32_t nframes, float* bkg_mesh,
                        float* rms_mesh, gp_stream stream);

/* ------------------------------------------------------- batched frames --
 * Several frames in one call.  The paper runs one frame per call; a frame of
 * a few megapixels leaves most of a GB300 idle, so here every stage runs as
 * one launch over all the frames of the call (grid y = frame).  Frames share
 * the parameters and the dtype; each has its own inputs, outputs and status
 * word, and its results are bit-identical to gp_extract's on that frame
 * alone (same kernels, same per-frame arithmetic and reduction order).
 *  - 1 <= n <= GP_MAX_BATCH; all frames GP_U16 or all GP_F32.
 *  - dp->nnear and dp->mask_out are not written (per-frame outputs that the
 *    batch does not carry).
 *  - net: NULL for the clipped estimator, else the learned background (one
 *    network pass over all frames when they share one mesh geometry).
 *  - Workspace: the sum of gp_workspace_bytes over the frames plus 256 KB
 *    suffices for the plain background.
 *  - Each frame's status word (device int32) must be zero on entry; after the
 *    stream completes it is 0 or the frame's first error (GP_ERR_CAPACITY:
 *    more segments than catalog rows; GP_ERR_TIMEOUT / GP_ERR_INTERNAL: see
 *    gp_ctx_sync).  The return value covers argument checks and launches. */
#define GP_MAX_BATCH 64
typedef struct {
    gp_image image;        /* device */
    gp_bkg bkg;            /* bkg_mesh, rms_mesh required (device); maps nullable */
    uint32_t* segmap;      /* device width*height */
    gp_catalog cat;        /* device columns and device count */
    double* flux;          /* device capacity*nr; nullable when nr = 0 or capacity = 0 */
    double* fluxerr;
    uint32_t* apflags;
    int32_t* status;       /* device word, zero on entry */
} gp_frame;

gp_status gp_extract_batch(gp_ctx* ctx, gp_frame* frames, int32_t n, const gp_bkg_params* bp,
                           const gp_det_params* dp, const gp_ap_params* ap, const gp_cnn_weights* net,
                           gp_stream stream);

/* --------------------------------------------------------- request server --
 * A long-lived loop that takes frames from host memory and returns their
 * catalogs, with continuous batching.  The paper processes one frame per
 * call and bounds how many frames run at once by device memory over a
 * frame's peak footprint (Section 6.4); the server makes that bound an
 * admission rule: a request is admitted when its device footprint (pixels,
 * segmentation map, workspace, results) fits the memory budget and an
 * execution slot is free, so frames that arrive while others run start as
 * soon as memory and a slot free up.  Small frames waiting together run as
 * one batched launch (gp_extract_batch); each slot has its own stream, so one
 * unit's host-to-device copy overlaps another's kernels.  A frame's results
 * are bit-identical to gp_extract's on it alone.
 *  - One worker thread owns all device work; submit, wait, release and stats
 *    may be called from any thread.
 *  - Requests are admitted in arrival order (a request that does not fit
 *    waits, and so do the ones behind it).
 *  - The request's host pixels must stay valid until its result is ready;
 *    pinned host memory lets the copy run asynchronously.
 *  - Results live in the server's pinned host memory until released. */
typedef struct gp_server gp_server;

typedef struct {
    int32_t device;
    size_t hbm_budget;        /* device bytes for work in flight (one allocation at create) */
    size_t host_budget;       /* pinned host bytes for results (one allocation at create) */
    int32_t slots;            /* units in flight at once, one stream each: 1 .. 16 */
    int64_t batch_pixels;     /* frames of at most this many pixels may share a launch */
    int32_t max_batch;        /* frames per launch, 1 .. GP_MAX_BATCH */
    gp_bkg_params bkg;
    gp_det_params det;        /* kernel taps copied at create; nnear and mask_out ignored */
    gp_ap_params ap;          /* radii copied at create */
    const gp_cnn_weights* net;  /* device weights (must outlive the server), or NULL: clipped estimator */
} gp_server_config;

typedef struct {
    gp_image image;           /* HOST pixels and optional host mask (pitch = width) */
    int32_t capacity;         /* catalog rows, >= 1 */
    int32_t want_segmap;      /* nonzero: copy the segmentation map back */
} gp_request;

typedef struct {
    int32_t status;           /* this frame's gp_status */
    int32_t n;                /* segments found; rows filled = min(n, capacity) */
    gp_catalog cat;           /* host columns (cat.n points at n), valid until release */
    const double* flux;       /* host capacity*nr */
    const double* fluxerr;
    const uint32_t* apflags;
    const uint32_t* segmap;   /* host width*height, or NULL */
    const float* bkg_mesh;    /* host my*mx */
    const float* rms_mesh;
    int32_t mesh, mx, my;
    int32_t batch;            /* frames in the launch this frame ran in */
    double latency_ms;        /* submit to result ready (host clock) */
    double queue_ms;          /* submit to admission */
    float h2d_ms;             /* the unit's input copies (device clock; shared by a batch's frames) */
    float run_ms;             /* the unit's pipeline kernels */
    float d2h_ms;             /* the unit's result copies */
} gp_result;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t units;            /* launches of the pipeline (a frame or a batch) */
    int64_t batched_frames;   /* frames that ran in a batch of two or more */
    double mpix;              /* megapixels of completed frames */
    double wall_s;            /* first submit to last completion */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* latency of completed frames */
    size_t budget, peak_bytes;                /* device budget and its peak use */
    int32_t peak_inflight;    /* most units in flight at once */
} gp_server_report;

gp_status gp_server_create(const gp_server_config* cfg, gp_server** out);
/* GP_ERR_OOM when the request could never fit the budgets */
gp_status gp_server_submit(gp_server* s, const gp_request* req, uint64_t* ticket);
/* the footprint the admission rule charges for this request run alone:
 * device bytes (pixels, mask, segmentation map, workspace, result block) and
 * pinned host bytes (result block, segmentation map if wanted) */
gp_status gp_server_request_bytes(const gp_server* s, const gp_request* req, size_t* device_bytes,
                                  size_t* host_bytes);
/* waits for the result (timeout_ms < 0: no limit; GP_ERR_TIMEOUT when it
 * expires first); returns the frame's own status */
gp_status gp_server_wait(gp_server* s, uint64_t ticket, int32_t timeout_ms, gp_result* out);
/* frees the result's host memory; its pointers become invalid */
gp_status gp_server_release(gp_server* s, uint64_t ticket);
/* counters and latency percentiles since create or the last reset */
gp_status gp_server_stats(gp_server* s, gp_server_report* out, int32_t reset);
/* finishes the work in flight, fails the requests not yet admitted, frees */
void gp_server_destroy(gp_server* s);

/* gp_background without a context, for callers that cannot allocate device
 * memory.  The paper has no counterpart.  Some callers must not call
 * cudaMalloc at all -- a
 * process whose device memory belongs to a pool it may not bypass, a plugin
 * loaded into an application that forbids allocations after start-up, a
 * latency-critical loop that must not take the allocator's locks -- and so
 * cannot create a gp_ctx, whose workspace is one cudaMalloc.  This entry
 * point allocates nothing: its scratch is a fixed array inside the library
 * image (about 172 KB, held on every GPU that loads the library until the
 * process exits).
 *  - Runs on the current device.  Same arguments and outputs as
 *    gp_background (caller-owned meshes and optional maps).
 *  - Limit: at most 3600 mesh boxes (ceil(width/mesh) * ceil(height/mesh));
 *    a larger mesh returns GP_ERR_INVALID_ARG with nothing enqueued.
 *  - The first call on a device looks up the scratch's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the rest of the
 *    process: it belongs to the device's primary context, so after a
 *    cudaDeviceReset, or on the device driven through another context, it is
 *    no longer valid and this entry point must not be called again.
 *  - Every call uses the same scratch, and each call rewrites all of it that
 *    it reads, so calls in sequence need nothing cleared; calls that overlap
 *    on the GPU (different streams, no ordering) race on it.
 *  - Errors are reported like gp_background's (gp_last_error()). */
gp_status gp_background_static(const gp_image* img, const gp_bkg_params* p, gp_bkg* bkg, gp_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GPPHOT_H */
