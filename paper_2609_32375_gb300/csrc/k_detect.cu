// k_detect.cu -- matched-filter detection and segmentation (paper Section
// 3.2, with labelled segments in place of the paper's local maxima).
//
//  k_detect_tile  one CTA per 64 x 32 tile.  Stages the tile plus a filter
//                 halo in shared memory as m = I - B (the spline background
//                 evaluated from per-column node rows), correlates it with
//                 the normalised kernel, thresholds F > k sigma(p), labels
//                 the tile's 8-connected components by union-find in shared
//                 memory (root = minimum index, i.e. the segment's first
//                 pixel in raster order) and writes the segmentation map.
//                 Components that do not touch an edge shared with another
//                 tile are final here; the others become "pieces" whose
//                 edge pixels are recorded for the merge.
//  k_merge        unites pieces across tile edges (lock-free union-find
//                 over piece ids, atomicMin linking).
//  k_aggregate    sums piece sizes, bounding boxes and minimum indices at
//                 each union-find root.
//  k_finalize     emits merged segments, and rewrites the map pixels of
//                 pieces whose final label differs (other root, or below
//                 minarea) -- a sparse pass over those pieces' boxes only.
//  k_rank_*       orders segments by label (bucket counts, one scan,
//                 scatter, in-bucket rank): a deterministic catalog order.
#include <math.h>

#include "gp_internal.cuh"
#include "gp_launch.h"

namespace gp {

constexpr int DT_NT = 256;
constexpr int KMAX = (2 * HMAX + 1) * (2 * HMAX + 1);

struct DetectArgs {
    float K[KMAX];            // normalised taps, kh rows of kw (kernel parameter space)
    Image im;
    SplineTab sb, sr;
    int kw, kh, hx, hy, hh;   // taps, half sizes, staged halo
    float thresh;
    int minarea;
    uint32_t* seg;
    uint8_t* mask_out;
    int* nnear;
    const uint8_t* in_mask;   // labelling of a given mask
    Tiles T;
    Pieces P;
    Comps C;
    int* status;
};

// ------------------------------------------------ shared-memory union-find ---
__device__ __forceinline__ int sfind(volatile int* lab, int x)
{
    for (int n = 0; n < TNPIX + 1; ++n) {
        int p = lab[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

__device__ __forceinline__ void sunite(int* lab, int a, int b)
{
    for (int it = 0; it < 4 * TNPIX; ++it) {
        a = sfind(lab, a);
        b = sfind(lab, b);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicMin(lab + a, b);
        if (old == a) return;
        a = old;
    }
}

// ---------------------------------------------------- global union-find ---
__device__ __forceinline__ int gfind(const int* parent, int x)
{
    for (int n = 0; n < WALK_LIMIT; ++n) {
        int p = __ldcg(parent + x);
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ void gunite(int* parent, int a, int b, int* status)
{
    for (int it = 0; it < WALK_LIMIT; ++it) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    set_status(status, GP_ERR_TIMEOUT);
}

// block-wide exclusive scan of one int per thread (DT_NT threads)
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < DT_NT / 32 ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < DT_NT / 32) warp_tot[lane] = wi - w;
        if (lane == DT_NT / 32 - 1) *total = wi;
    }
    __syncthreads();
    int r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

template <bool F32, bool LABEL_ONLY>
__global__ void __launch_bounds__(DT_NT) k_detect_tile(DetectArgs A)
{
    // m over tile + halo; reused after thresholding for per-root records
    __shared__ __align__(16) float sm_m[SH * SW];
    __shared__ int lab[TNPIX];
    __shared__ __align__(16) uint8_t badpx[TNPIX];   // reused as root pixel list
    __shared__ short rid[TNPIX];
    __shared__ float4 colv[NJMAX * SW];   // per column and node row: (u_bkg, w_bkg, u_rms, w_rms)
    __shared__ float4 rowc[SH];            // per staged row: (b, c0, c1, -)
    __shared__ int2 rowj[SH];
    __shared__ int jlo_s, jhi_s;
    __shared__ int warp_tot[DT_NT / 32];
    __shared__ int nroots_s, npieces_s, ncomps_s, pbase_s, cbase_s;
    __shared__ int near_s;

    int* r_val = reinterpret_cast<int*>(sm_m);          // value written to the map
    int* r_xmin = r_val + MAXROOT;
    int* r_xmax = r_xmin + MAXROOT;
    int* r_ymin = r_xmax + MAXROOT;
    int* r_ymax = r_ymin + MAXROOT;
    int* r_pidx = r_ymax + MAXROOT;                     // border flag, then local piece index
    int* r_pix = reinterpret_cast<int*>(badpx);         // root's tile pixel

    const int tid = threadIdx.x;
    const int W = A.im.W, H = A.im.H;
    const int tile = blockIdx.x;
    const int ntx = A.T.ntx;
    const int tx = tile % ntx, ty = tile / ntx;
    const int x0 = tx * TX, y0 = ty * TY;
    const int tw = min(TX, W - x0), th = min(TY, H - y0);

    if (!LABEL_ONLY) {
        const int hh = A.hh;
        const int scols = tw + 2 * hh, srows = th + 2 * hh;
        if (tid == 0) { jlo_s = 1 << 30; jhi_s = -1; near_s = 0; }
        __syncthreads();
        // node rows needed by the staged rows
        for (int ry = tid; ry < srows; ry += DT_NT) {
            int gy = mirror_idx(y0 - hh + ry, H);
            AxCoef c = axis_coef(A.sb.ay, (float)gy);
            atomicMin(&jlo_s, c.i);
            atomicMax(&jhi_s, c.i1);
        }
        __syncthreads();
        const int jlo = jlo_s;
        const int nj = jhi_s - jlo + 1;
        if (nj > NJMAX) {   // excluded by the host's mesh >= 16 rule
            if (tid == 0) set_status(A.status, GP_ERR_INTERNAL);
            return;
        }
        for (int ry = tid; ry < srows; ry += DT_NT) {
            int gy = mirror_idx(y0 - hh + ry, H);
            AxCoef c = axis_coef(A.sb.ay, (float)gy);
            rowc[ry] = make_float4(c.b, c.c0, c.c1, 0.f);
            rowj[ry] = make_int2(c.i - jlo, c.i1 - jlo);
        }
        for (int q = tid; q < nj * scols; q += DT_NT) {
            int jj = q / scols, cx = q - jj * scols;
            int gx = mirror_idx(x0 - hh + cx, W);
            AxCoef c = axis_coef(A.sb.ax, (float)gx);
            float2 b = row_eval(A.sb, jlo + jj, c);
            float2 r = row_eval(A.sr, jlo + jj, c);
            colv[jj * SW + cx] = make_float4(b.x, b.y, r.x, r.y);
        }
        __syncthreads();
        // stage m = I - B over tile + halo (mirror border; bad pixels -> 0)
        for (int q = tid; q < srows * scols; q += DT_NT) {
            int ry = q / scols, cx = q - ry * scols;
            int gx = mirror_idx(x0 - hh + cx, W), gy = mirror_idx(y0 - hh + ry, H);
            float v;
            bool bad;
            if (F32) {
                v = __ldg(reinterpret_cast<const float*>(A.im.data) + (int64_t)gy * A.im.pitch + gx);
                bad = !isfinite(v);
            } else {
                v = (float)__ldg(reinterpret_cast<const uint16_t*>(A.im.data) + (int64_t)gy * A.im.pitch + gx);
                bad = false;
            }
            if (A.im.mask && A.im.mask[(int64_t)gy * W + gx]) bad = true;
            int2 j = rowj[ry];
            float4 c = rowc[ry];
            float4 n0 = colv[j.x * SW + cx], n1 = colv[j.y * SW + cx];
            AxCoef cy; cy.b = c.x; cy.c0 = c.y; cy.c1 = c.z;
            float Bv = axis_combine(cy, n0.x, n1.x, n0.y, n1.y);
            sm_m[ry * SW + cx] = bad ? 0.f : v - Bv;
            int py = ry - hh, px = cx - hh;
            if (py >= 0 && py < th && px >= 0 && px < tw) badpx[py * TX + px] = bad;
        }
        __syncthreads();
        // matched filter, threshold
        int nnear = 0;
        for (int p = tid; p < TNPIX; p += DT_NT) {
            int py = p / TX, px = p - py * TX;
            bool fg = false;
            if (py < th && px < tw) {
                float F = 0.f;
                const int r0 = py + hh - A.hy, c0 = px + hh - A.hx;
                for (int v = 0; v < A.kh; ++v) {
                    const float* row = sm_m + (r0 + v) * SW + c0;
                    const float* kr = A.K + v * A.kw;
                    for (int u = 0; u < A.kw; ++u) F = fmaf(kr[u], row[u], F);
                }
                int ry = py + hh, cx = px + hh;
                int2 j = rowj[ry];
                float4 c = rowc[ry];
                float4 n0 = colv[j.x * SW + cx], n1 = colv[j.y * SW + cx];
                AxCoef cy; cy.b = c.x; cy.c0 = c.y; cy.c1 = c.z;
                float sig = axis_combine(cy, n0.z, n1.z, n0.w, n1.w);
                float thr = A.thresh * sig;
                fg = (F > thr) && !badpx[p];
                if (fabsf(F - thr) <= 1e-5f * fabsf(thr)) ++nnear;
                if (A.mask_out) A.mask_out[(int64_t)(y0 + py) * W + x0 + px] = fg ? 1 : 0;
            }
            lab[p] = fg ? p : -1;
        }
        if (A.nnear) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nnear += __shfl_xor_sync(0xffffffffu, nnear, o);
            if ((tid & 31) == 0 && nnear) atomicAdd(&near_s, nnear);
        }
        __syncthreads();
        if (A.nnear && tid == 0 && near_s) atomicAdd(A.nnear, near_s);
    } else {
        for (int p = tid; p < TNPIX; p += DT_NT) {
            int py = p / TX, px = p - py * TX;
            bool fg = py < th && px < tw && A.in_mask[(int64_t)(y0 + py) * W + x0 + px] != 0;
            lab[p] = fg ? p : -1;
        }
        __syncthreads();
    }

    // ---- tile-local union-find: link each pixel to its W, NW, N, NE neighbours
    for (int p = tid; p < TNPIX; p += DT_NT) {
        if (lab[p] < 0) continue;
        int py = p / TX, px = p - py * TX;
        if (px > 0 && lab[p - 1] >= 0) sunite(lab, p, p - 1);
        if (py > 0) {
            if (px > 0 && lab[p - TX - 1] >= 0) sunite(lab, p, p - TX - 1);
            if (lab[p - TX] >= 0) sunite(lab, p, p - TX);
            if (px + 1 < tw && lab[p - TX + 1] >= 0) sunite(lab, p, p - TX + 1);
        }
    }
    __syncthreads();
    for (int p = tid; p < TNPIX; p += DT_NT)
        if (lab[p] >= 0) lab[p] = sfind(lab, p);
    __syncthreads();

    // ---- compact root numbering in raster (= label) order
    {
        const int per = TNPIX / DT_NT;   // 8 contiguous pixels per thread
        int cnt = 0;
        for (int e = 0; e < per; ++e) {
            int p = tid * per + e;
            cnt += (lab[p] == p);
        }
        int off = block_excl_scan(cnt, warp_tot, &nroots_s);
        for (int e = 0; e < per; ++e) {
            int p = tid * per + e;
            if (lab[p] == p) {
                rid[p] = (short)off;
                r_pix[off] = p;
                ++off;
            }
        }
    }
    __syncthreads();
    const int nroots = nroots_s;
    for (int r = tid; r < nroots; r += DT_NT) {
        r_val[r] = 0; r_xmin[r] = TX; r_xmax[r] = -1; r_ymin[r] = TY; r_ymax[r] = -1; r_pidx[r] = 0;
    }
    __syncthreads();
    for (int p = tid; p < TNPIX; p += DT_NT) {
        int l = lab[p];
        if (l < 0) continue;
        int r = rid[l];
        int py = p / TX, px = p - py * TX;
        atomicAdd(r_val + r, 1);
        atomicMin(r_xmin + r, px); atomicMax(r_xmax + r, px);
        atomicMin(r_ymin + r, py); atomicMax(r_ymax + r, py);
        bool border = (px == 0 && x0 > 0) || (px == tw - 1 && x0 + tw < W) ||
                      (py == 0 && y0 > 0) || (py == th - 1 && y0 + th < H);
        if (border) r_pidx[r] = 1;
    }
    __syncthreads();

    // ---- decide: pieces (touch a shared tile edge), final segments, dropped
    int isp[2], isc[2];
    int pc = 0, cc = 0;
    for (int e = 0; e < 2; ++e) {
        int r = tid * 2 + e;
        isp[e] = (r < nroots) && r_pidx[r];
        isc[e] = (r < nroots) && !r_pidx[r] && r_val[r] >= A.minarea;
        pc += isp[e]; cc += isc[e];
    }
    int poff = block_excl_scan(pc, warp_tot, &npieces_s);
    int coff = block_excl_scan(cc, warp_tot, &ncomps_s);
    if (tid == 0) {
        pbase_s = npieces_s ? atomicAdd(A.P.count, npieces_s) : 0;
        cbase_s = ncomps_s ? atomicAdd(A.C.count, ncomps_s) : 0;
        A.T.piece_base[tile] = pbase_s;
        A.T.piece_cnt[tile] = npieces_s;
    }
    __syncthreads();
    const int pbase = pbase_s, cbase = cbase_s;
    for (int e = 0; e < 2; ++e) {
        int r = tid * 2 + e;
        if (r >= nroots) continue;
        int p = r_pix[r];
        int py = p / TX, px = p - py * TX;
        uint32_t L = (uint32_t)(y0 + py) * (uint32_t)W + (uint32_t)(x0 + px);
        int4 bb = make_int4(x0 + r_xmin[r], x0 + r_xmax[r], y0 + r_ymin[r], y0 + r_ymax[r]);
        int npix = r_val[r];
        int val = 0, pidx = -1;
        if (isp[e]) {
            int id = pbase + poff;
            if (id < A.P.cap) {
                A.P.root[id] = L; A.P.npix[id] = npix; A.P.bbox[id] = bb; A.P.parent[id] = id;
                A.P.agg_min[id] = L; A.P.agg_npix[id] = npix; A.P.agg_bbox[id] = bb;
                pidx = poff;
            } else {
                set_status(A.status, GP_ERR_INTERNAL);
            }
            val = (int)(L + 1u);
            ++poff;
        } else if (isc[e]) {
            int id = cbase + coff;
            if (id < A.C.cap) {
                A.C.label[id] = L + 1u; A.C.npix[id] = npix; A.C.bbox[id] = bb;
            } else {
                set_status(A.status, GP_ERR_INTERNAL);
            }
            val = (int)(L + 1u);
            ++coff;
        }
        r_val[r] = val;
        r_pidx[r] = pidx;
    }
    __syncthreads();

    // ---- segmentation map for the tile (coalesced rows)
    for (int p = tid; p < TNPIX; p += DT_NT) {
        int py = p / TX, px = p - py * TX;
        if (py >= th || px >= tw) continue;
        int l = lab[p];
        uint32_t v = l >= 0 ? (uint32_t)r_val[rid[l]] : 0u;
        A.seg[(int64_t)(y0 + py) * W + x0 + px] = v;
    }
    // ---- edge records: local piece index of each edge pixel, or -1
    int16_t* ed = A.T.edges + (int64_t)tile * EDGE_PER_TILE;
    for (int q = tid; q < EDGE_PER_TILE; q += DT_NT) {
        int px, py;
        bool ok;
        if (q < TY) { py = q; px = 0; ok = py < th; }                                   // colL
        else if (q < 2 * TY) { py = q - TY; px = tw - 1; ok = py < th; }               // colR
        else if (q < 2 * TY + TX) { px = q - 2 * TY; py = 0; ok = px < tw; }           // rowT
        else { px = q - 2 * TY - TX; py = th - 1; ok = px < tw; }                      // rowB
        int16_t v = -1;
        if (ok) {
            int l = lab[py * TX + px];
            if (l >= 0) v = (int16_t)r_pidx[rid[l]];
        }
        ed[q] = v;
    }
}

// ------------------------------------------------------------ tile merge ---
__global__ void k_merge(Tiles T, Pieces P, int W, int H, int* status)
{
    const int tile = blockIdx.x;
    const int ntx = T.ntx, nty = T.nty;
    const int tx = tile % ntx, ty = tile / ntx;
    const int tw = min(TX, W - tx * TX), th = min(TY, H - ty * TY);
    if (threadIdx.x == 0 && tx + 1 < ntx && ty + 1 < nty) {
        // anti-diagonal across this tile's bottom-right corner: bottom-left
        // pixel of the right tile and top-right pixel of the tile below
        // (independent of whether this tile has pieces)
        const int rt = tile + 1, dn = tile + ntx;
        if (T.piece_cnt[rt] > 0 && T.piece_cnt[dn] > 0) {
            int a = T.edges[(int64_t)rt * EDGE_PER_TILE + th - 1];
            int b = T.edges[(int64_t)dn * EDGE_PER_TILE + TY + 0];
            if (a >= 0 && b >= 0) gunite(P.parent, T.piece_base[rt] + a, T.piece_base[dn] + b, status);
        }
    }
    if (T.piece_cnt[tile] == 0) return;
    const int base = T.piece_base[tile];
    const int16_t* e = T.edges + (int64_t)tile * EDGE_PER_TILE;
    if (tx + 1 < ntx && T.piece_cnt[tile + 1] > 0) {
        const int nbase = T.piece_base[tile + 1];
        const int16_t* en = T.edges + (int64_t)(tile + 1) * EDGE_PER_TILE;
        for (int i = threadIdx.x; i < th; i += blockDim.x) {
            int a = e[TY + i];
            if (a < 0) continue;
            for (int d = -1; d <= 1; ++d) {
                int k = i + d;
                if (k < 0 || k >= th) continue;
                int b = en[k];
                if (b >= 0) gunite(P.parent, base + a, nbase + b, status);
            }
        }
    }
    if (ty + 1 < nty && T.piece_cnt[tile + ntx] > 0) {
        const int nbase = T.piece_base[tile + ntx];
        const int16_t* en = T.edges + (int64_t)(tile + ntx) * EDGE_PER_TILE;
        for (int j = threadIdx.x; j < tw; j += blockDim.x) {
            int a = e[2 * TY + TX + j];
            if (a < 0) continue;
            for (int d = -1; d <= 1; ++d) {
                int k = j + d;
                if (k < 0 || k >= tw) continue;
                int b = en[2 * TY + k];
                if (b >= 0) gunite(P.parent, base + a, nbase + b, status);
            }
        }
    }
    if (threadIdx.x == 0 && tx + 1 < ntx && ty + 1 < nty) {
        // bottom-right pixel of this tile and top-left pixel of the diagonal tile
        const int dr = tile + ntx + 1;
        int a = e[TY + th - 1];
        int b = T.edges[(int64_t)dr * EDGE_PER_TILE + 0];
        if (a >= 0 && b >= 0) gunite(P.parent, base + a, T.piece_base[dr] + b, status);
    }
}

// --------------------------------------------------------- piece resolve ---
__global__ void k_aggregate(Pieces P, int* status)
{
    const int n = min(*P.count, P.cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int r = gfind(P.parent, p);
        if (r < 0) { set_status(status, GP_ERR_TIMEOUT); continue; }
        if (r == p) continue;
        atomicMin(P.agg_min + r, P.root[p]);
        atomicAdd(P.agg_npix + r, P.npix[p]);
        int4 b = P.bbox[p];
        int* ab = reinterpret_cast<int*>(P.agg_bbox + r);
        atomicMin(ab + 0, b.x); atomicMax(ab + 1, b.y);
        atomicMin(ab + 2, b.z); atomicMax(ab + 3, b.w);
    }
}

// one warp per piece: emit merged segments at root pieces; rewrite the map
// pixels of pieces whose final label differs from their provisional one
__global__ void k_finalize(Pieces P, Comps C, uint32_t* seg, int W, int minarea, int* status)
{
    const int n = min(*P.count, P.cap);
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int p = wid; p < n; p += nw) {
        int r = gfind(P.parent, p);
        if (r < 0) { if (lane == 0) set_status(status, GP_ERR_TIMEOUT); continue; }
        int tot = P.agg_npix[r];
        uint32_t fin = tot >= minarea ? P.agg_min[r] + 1u : 0u;
        if (r == p && fin && lane == 0) {
            int id = atomicAdd(C.count, 1);
            if (id < C.cap) {
                C.label[id] = fin; C.npix[id] = tot; C.bbox[id] = P.agg_bbox[r];
            } else {
                set_status(status, GP_ERR_INTERNAL);
            }
        }
        uint32_t prov = P.root[p] + 1u;
        if (fin == prov) continue;
        int4 b = P.bbox[p];
        int bw = b.y - b.x + 1, bh = b.w - b.z + 1;
        for (int q = lane; q < bw * bh; q += 32) {
            int y = b.z + q / bw, x = b.x + q % bw;
            uint32_t* s = seg + (int64_t)y * W + x;
            if (*s == prov) *s = fin;
        }
    }
}

// ------------------------------------------------------------------ rank ---
__global__ void k_rank_count(Comps C)
{
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        atomicAdd(C.bcnt + ((C.label[c] - 1u) >> C.shift), 1);
}

constexpr int SCAN_NT = 1024;

// exclusive scan of the bucket counts (one CTA); publishes the segment count
__global__ void __launch_bounds__(SCAN_NT) k_rank_scan(Comps C, int* n_out, int capacity, int* status)
{
    __shared__ int wsum[SCAN_NT / 32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < C.nb; base += SCAN_NT) {
        int i = base + tid;
        int v = i < C.nb ? C.bcnt[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        int excl = carry + wsum[warp] + incl - v;
        if (i < C.nb) C.boff[i] = excl;
        __syncthreads();
        if (tid == SCAN_NT - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) {
        int total = *C.count;
        if (total > C.cap) set_status(status, GP_ERR_INTERNAL);
        if (n_out) *n_out = total;
        if (capacity >= 0 && total > capacity) set_status(status, GP_ERR_CAPACITY);
    }
}

__global__ void k_rank_scatter(Comps C)
{
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int b = (int)((C.label[c] - 1u) >> C.shift);
        int s = C.boff[b] + atomicAdd(C.bcur + b, 1);
        C.slots[s] = c;
    }
}

__global__ void k_rank_place(Comps C)
{
    const int n = min(*C.count, C.cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        uint32_t l = C.label[c];
        int b = (int)((l - 1u) >> C.shift);
        int s0 = C.boff[b], s1 = s0 + C.bcnt[b];
        int r = s0;
        for (int s = s0; s < s1; ++s) r += (C.label[C.slots[s]] < l);
        C.perm[r] = c;
    }
}

// --------------------------------------------------------------- launchers ---
cudaError_t launch_detect_tiles(const Image& im, const SplineTab& sb, const SplineTab& sr, const float* taps,
                                int kw, int kh, float thresh, int minarea, uint32_t* seg, uint8_t* mask_out, int* nnear,
                                const uint8_t* in_mask, const Tiles& T, const Pieces& P, const Comps& C,
                                int* status, cudaStream_t st)
{
    DetectArgs A;
    for (int i = 0; i < KMAX; ++i) A.K[i] = (taps && i < kw * kh) ? taps[i] : 0.f;
    A.im = im; A.sb = sb; A.sr = sr;
    A.kw = kw; A.kh = kh; A.hx = kw / 2; A.hy = kh / 2; A.hh = max(kw / 2, kh / 2);
    A.thresh = thresh; A.minarea = minarea;
    A.seg = seg; A.mask_out = mask_out; A.nnear = nnear; A.in_mask = in_mask;
    A.T = T; A.P = P; A.C = C; A.status = status;
    const int ntiles = T.ntx * T.nty;
    if (in_mask)
        k_detect_tile<false, true><<<ntiles, DT_NT, 0, st>>>(A);
    else if (im.is_f32)
        k_detect_tile<true, false><<<ntiles, DT_NT, 0, st>>>(A);
    else
        k_detect_tile<false, false><<<ntiles, DT_NT, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const Tiles& T, const Pieces& P, const Comps& C, uint32_t* seg, int W, int H,
                           int minarea, int* status, cudaStream_t st)
{
    const int ntiles = T.ntx * T.nty;
    k_merge<<<ntiles, 64, 0, st>>>(T, P, W, H, status);
    const int g = 152 * 8;
    k_aggregate<<<g, 256, 0, st>>>(P, status);
    k_finalize<<<g, 256, 0, st>>>(P, C, seg, W, minarea, status);
    return cudaGetLastError();
}

cudaError_t launch_rank(const Comps& C, int* n_out, int capacity, bool place, int* status, cudaStream_t st)
{
    const int g = 152 * 4;
    k_rank_count<<<g, 256, 0, st>>>(C);
    k_rank_scan<<<1, SCAN_NT, 0, st>>>(C, n_out, capacity, status);
    if (place) {
        k_rank_scatter<<<g, 256, 0, st>>>(C);
        k_rank_place<<<g, 256, 0, st>>>(C);
    }
    return cudaGetLastError();
}

}  // namespace gp
