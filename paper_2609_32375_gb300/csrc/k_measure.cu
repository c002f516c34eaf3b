// k_measure.cu -- catalog rows and circular apertures with exact disc/pixel
// overlap areas (paper Section 3.4).
//
// One warp per source.  The segment moments were finished after detection
// (k_mom_finish); here the apertures scan the pixels around the centroid once
// for all radii, leaving raw sums that k_ap_finish_rows / k_ap_finish_list
// finish one result per thread (k_ap_finish_rows also writes each catalog
// row, in label order).  Every sum is a float-float
// (compensated) accumulation of FP32 products, reduced across the warp in a
// fixed butterfly order, so results are reproducible run to run and carry
// about 48 bits -- the float64-class accumulation the paper asks of aperture
// sums, without FP64 arithmetic (which runs at a small fraction of the FP32
// rate on this GPU).
#include "k_measure_impl.cuh"

namespace gp {

// --------------------------------------------------------------- launchers ---
static ApSpec make_ap(const float* radii, int nr, float gain)
{
    ApSpec s;
    s.nr = nr;
    s.rmax = 0.f;
    for (int k = 0; k < MAX_NR; ++k) {
        s.r[k] = k < nr ? radii[k] : 0.f;
        if (k < nr) s.rmax = fmaxf(s.rmax, radii[k]);
    }
    s.gain = gain;
    s.inv_gain = gain > 0.f ? 1.0 / (double)gain : 0.0;
    return s;
}

MeasureArgs measure_args(const Image& im, const SplineTab& sb, const SplineTab& sr, const Comps& C,
                         const gp_catalog& cat, const float* radii, int nr, float gain, double* apflux,
                         double* apferr, uint32_t* apflags)
{
    MeasureArgs A;
    A.im = im; A.sb = sb; A.sr = sr; A.C = C;
    A.capacity = cat.capacity;
    A.label = cat.label; A.npix = cat.npix; A.flux_iso = cat.flux_iso;
    A.x = cat.x; A.y = cat.y; A.x2 = cat.x2; A.y2 = cat.y2; A.xy = cat.xy;
    A.xmin = cat.xmin; A.xmax = cat.xmax; A.ymin = cat.ymin; A.ymax = cat.ymax;
    A.peak = cat.peak; A.xpeak = cat.xpeak; A.ypeak = cat.ypeak; A.flags = cat.flags;
    A.ap = make_ap(radii, nr, gain);
    A.apflux = apflux; A.apferr = apferr; A.apflags = apflags;
    return A;
}

// every frame of a batch shares `one`'s dtype and number of radii
cudaError_t launch_measure_any(const MeasureArgs& one, const MeasureArgs* batch, int nframes, cudaStream_t st)
{
    // exactly the resident CTAs (3 per SM at the kernel's launch bounds): the
    // warps' grid-stride loops share the sources with no partial last wave
    int g = 152 * 3 / nframes;
    if (g < 16) g = 16;
    const dim3 grid(g, nframes);
    if (batch) return launch_measure_batched(one, batch, grid, st);
    if (one.ap.nr > 0) {
        const cudaError_t e = one.im.is_f32 ? dispatch_nr<MeasureLaunch, true>(one.ap.nr, one, grid, st)
                                            : dispatch_nr<MeasureLaunch, false>(one.ap.nr, one, grid, st);
        if (e != cudaSuccess) return e;
    }
    launch_dep(k_ap_finish_rows<false>, grid, dim3(256), 0, st, (const MeasureArgs*)nullptr, one);
    return cudaGetLastError();
}

cudaError_t launch_measure(const Image& im, const SplineTab& sb, const SplineTab& sr, const Comps& C,
                           const uint32_t* seg, const gp_catalog& cat, const float* radii, int nr, float gain,
                           double* apflux, double* apferr, uint32_t* apflags, cudaStream_t st)
{
    (void)seg;
    return launch_measure_any(measure_args(im, sb, sr, C, cat, radii, nr, gain, apflux, apferr, apflags), nullptr, 1,
                              st);
}

cudaError_t launch_aperture(const Image& im, const SplineTab& sb, const SplineTab& sr, const double* xs,
                            const double* ys, int n, const float* radii, int nr, float gain, double* flux,
                            double* ferr, uint32_t* fl, cudaStream_t st)
{
    ApSpec ap = make_ap(radii, nr, gain);
    int64_t g64 = ((int64_t)n * 32 + 255) / 256;
    int g = (int)(g64 < 152 * 3 ? g64 : 152 * 3);
    if (g < 1) g = 1;
    if (im.is_f32) return dispatch_nr<ApertureLaunch, true>(nr, im, sb, sr, ap, xs, ys, n, flux, ferr, fl, g, st);
    return dispatch_nr<ApertureLaunch, false>(nr, im, sb, sr, ap, xs, ys, n, flux, ferr, fl, g, st);
}

}  // namespace gp
