// median_sel.cuh -- written by gen_median.py (do not edit): median-selection
// networks pruned from Batcher's odd-even merge sort (see gen_median.py).
// med_sel<N>(v) returns the middle value of v[0 .. N-1] (N odd, no NaN);
// v is overwritten.
#pragma once

namespace gp {

template <int N>
__device__ __forceinline__ float med_sel(float (&v)[N]);

// 9 values: 24 comparators, 16 of them full compare-exchanges
template <>
__device__ __forceinline__ float med_sel<9>(float (&v)[9])
{
    { const float a = v[0], b = v[1]; v[0] = fminf(a, b); v[1] = fmaxf(a, b); }
    { const float a = v[2], b = v[3]; v[2] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[0], b = v[2]; v[0] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[1], b = v[3]; v[1] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[4], b = v[5]; v[4] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[6], b = v[7]; v[6] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[4], b = v[6]; v[4] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[5], b = v[7]; v[5] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[0], b = v[4]; v[0] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[2], b = v[6]; v[2] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[1], b = v[5]; v[1] = fminf(a, b); v[5] = fmaxf(a, b); }
    v[3] = fminf(v[3], v[7]);
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    v[2] = fmaxf(v[1], v[2]);
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    v[5] = fminf(v[5], v[6]);
    v[8] = fmaxf(v[0], v[8]);
    v[4] = fminf(v[4], v[8]);
    v[4] = fmaxf(v[2], v[4]);
    v[3] = fminf(v[3], v[5]);
    v[4] = fmaxf(v[3], v[4]);
    return v[4];
}

// 25 values: 113 comparators, 89 of them full compare-exchanges
template <>
__device__ __forceinline__ float med_sel<25>(float (&v)[25])
{
    { const float a = v[0], b = v[1]; v[0] = fminf(a, b); v[1] = fmaxf(a, b); }
    { const float a = v[2], b = v[3]; v[2] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[0], b = v[2]; v[0] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[1], b = v[3]; v[1] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[4], b = v[5]; v[4] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[6], b = v[7]; v[6] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[4], b = v[6]; v[4] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[5], b = v[7]; v[5] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[0], b = v[4]; v[0] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[2], b = v[6]; v[2] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[1], b = v[5]; v[1] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[3], b = v[7]; v[3] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[8], b = v[9]; v[8] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[10], b = v[11]; v[10] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[8], b = v[10]; v[8] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[9], b = v[11]; v[9] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[12], b = v[13]; v[12] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[14], b = v[15]; v[14] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[12], b = v[14]; v[12] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[13], b = v[15]; v[13] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[8], b = v[12]; v[8] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[10], b = v[14]; v[10] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[10], b = v[12]; v[10] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[9], b = v[13]; v[9] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[11], b = v[15]; v[11] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[11], b = v[13]; v[11] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[11], b = v[12]; v[11] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[0], b = v[8]; v[0] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[4], b = v[12]; v[4] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[4], b = v[8]; v[4] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[2], b = v[10]; v[2] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[6], b = v[14]; v[6] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[6], b = v[10]; v[6] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[6], b = v[8]; v[6] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[10], b = v[12]; v[10] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[1], b = v[9]; v[1] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[5], b = v[13]; v[5] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[5], b = v[9]; v[5] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[3], b = v[11]; v[3] = fminf(a, b); v[11] = fmaxf(a, b); }
    v[7] = fminf(v[7], v[15]);
    { const float a = v[7], b = v[11]; v[7] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[7], b = v[9]; v[7] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[11], b = v[13]; v[11] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[7], b = v[8]; v[7] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[11], b = v[12]; v[11] = fminf(a, b); v[12] = fmaxf(a, b); }
    v[13] = fminf(v[13], v[14]);
    { const float a = v[16], b = v[17]; v[16] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[18], b = v[19]; v[18] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[16], b = v[18]; v[16] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[17], b = v[19]; v[17] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[20], b = v[21]; v[20] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[22], b = v[23]; v[22] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[20], b = v[22]; v[20] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[21], b = v[23]; v[21] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[16], b = v[20]; v[16] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[18], b = v[22]; v[18] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[18], b = v[20]; v[18] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[17], b = v[21]; v[17] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[19], b = v[23]; v[19] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[19], b = v[21]; v[19] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[19], b = v[20]; v[19] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[16], b = v[24]; v[16] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[20], b = v[24]; v[20] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[18], b = v[20]; v[18] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[22], b = v[24]; v[22] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[19], b = v[21]; v[19] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[19], b = v[20]; v[19] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[23], b = v[24]; v[23] = fminf(a, b); v[24] = fmaxf(a, b); }
    v[16] = fmaxf(v[0], v[16]);
    v[8] = fminf(v[8], v[24]);
    v[16] = fmaxf(v[8], v[16]);
    v[20] = fmaxf(v[4], v[20]);
    v[12] = fminf(v[12], v[20]);
    v[12] = fminf(v[12], v[16]);
    v[18] = fmaxf(v[2], v[18]);
    v[10] = fminf(v[10], v[18]);
    v[6] = fminf(v[6], v[22]);
    v[10] = fmaxf(v[6], v[10]);
    v[12] = fmaxf(v[10], v[12]);
    v[17] = fmaxf(v[1], v[17]);
    v[17] = fmaxf(v[9], v[17]);
    v[21] = fmaxf(v[5], v[21]);
    v[13] = fminf(v[13], v[21]);
    v[13] = fminf(v[13], v[17]);
    v[19] = fmaxf(v[3], v[19]);
    v[11] = fminf(v[11], v[19]);
    v[7] = fminf(v[7], v[23]);
    v[11] = fmaxf(v[7], v[11]);
    v[11] = fminf(v[11], v[13]);
    v[12] = fmaxf(v[11], v[12]);
    return v[12];
}

// 49 values: 319 comparators, 271 of them full compare-exchanges
template <>
__device__ __forceinline__ float med_sel<49>(float (&v)[49])
{
    { const float a = v[0], b = v[1]; v[0] = fminf(a, b); v[1] = fmaxf(a, b); }
    { const float a = v[2], b = v[3]; v[2] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[0], b = v[2]; v[0] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[1], b = v[3]; v[1] = fminf(a, b); v[3] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[4], b = v[5]; v[4] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[6], b = v[7]; v[6] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[4], b = v[6]; v[4] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[5], b = v[7]; v[5] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[0], b = v[4]; v[0] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[2], b = v[6]; v[2] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[1], b = v[5]; v[1] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[3], b = v[7]; v[3] = fminf(a, b); v[7] = fmaxf(a, b); }
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[8], b = v[9]; v[8] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[10], b = v[11]; v[10] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[8], b = v[10]; v[8] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[9], b = v[11]; v[9] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[12], b = v[13]; v[12] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[14], b = v[15]; v[14] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[12], b = v[14]; v[12] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[13], b = v[15]; v[13] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[8], b = v[12]; v[8] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[10], b = v[14]; v[10] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[10], b = v[12]; v[10] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[9], b = v[13]; v[9] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[11], b = v[15]; v[11] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[11], b = v[13]; v[11] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[11], b = v[12]; v[11] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[0], b = v[8]; v[0] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[4], b = v[12]; v[4] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[4], b = v[8]; v[4] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[2], b = v[10]; v[2] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[6], b = v[14]; v[6] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[6], b = v[10]; v[6] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[6], b = v[8]; v[6] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[10], b = v[12]; v[10] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[1], b = v[9]; v[1] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[5], b = v[13]; v[5] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[5], b = v[9]; v[5] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[3], b = v[11]; v[3] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[7], b = v[15]; v[7] = fminf(a, b); v[15] = fmaxf(a, b); }
    { const float a = v[7], b = v[11]; v[7] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[7], b = v[9]; v[7] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[11], b = v[13]; v[11] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[7], b = v[8]; v[7] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[11], b = v[12]; v[11] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[16], b = v[17]; v[16] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[18], b = v[19]; v[18] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[16], b = v[18]; v[16] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[17], b = v[19]; v[17] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[20], b = v[21]; v[20] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[22], b = v[23]; v[22] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[20], b = v[22]; v[20] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[21], b = v[23]; v[21] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[16], b = v[20]; v[16] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[18], b = v[22]; v[18] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[18], b = v[20]; v[18] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[17], b = v[21]; v[17] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[19], b = v[23]; v[19] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[19], b = v[21]; v[19] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[19], b = v[20]; v[19] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[24], b = v[25]; v[24] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[26], b = v[27]; v[26] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[24], b = v[26]; v[24] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[25], b = v[27]; v[25] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[25], b = v[26]; v[25] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[28], b = v[29]; v[28] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[30], b = v[31]; v[30] = fminf(a, b); v[31] = fmaxf(a, b); }
    { const float a = v[28], b = v[30]; v[28] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[29], b = v[31]; v[29] = fminf(a, b); v[31] = fmaxf(a, b); }
    { const float a = v[29], b = v[30]; v[29] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[24], b = v[28]; v[24] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[26], b = v[30]; v[26] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[26], b = v[28]; v[26] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[25], b = v[29]; v[25] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[27], b = v[31]; v[27] = fminf(a, b); v[31] = fmaxf(a, b); }
    { const float a = v[27], b = v[29]; v[27] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[25], b = v[26]; v[25] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[27], b = v[28]; v[27] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[29], b = v[30]; v[29] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[16], b = v[24]; v[16] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[20], b = v[28]; v[20] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[20], b = v[24]; v[20] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[18], b = v[26]; v[18] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[22], b = v[30]; v[22] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[22], b = v[26]; v[22] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[18], b = v[20]; v[18] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[22], b = v[24]; v[22] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[26], b = v[28]; v[26] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[17], b = v[25]; v[17] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[21], b = v[29]; v[21] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[21], b = v[25]; v[21] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[19], b = v[27]; v[19] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[23], b = v[31]; v[23] = fminf(a, b); v[31] = fmaxf(a, b); }
    { const float a = v[23], b = v[27]; v[23] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[19], b = v[21]; v[19] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[23], b = v[25]; v[23] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[27], b = v[29]; v[27] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[19], b = v[20]; v[19] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[23], b = v[24]; v[23] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[25], b = v[26]; v[25] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[27], b = v[28]; v[27] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[29], b = v[30]; v[29] = fminf(a, b); v[30] = fmaxf(a, b); }
    { const float a = v[0], b = v[16]; v[0] = fminf(a, b); v[16] = fmaxf(a, b); }
    { const float a = v[8], b = v[24]; v[8] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[8], b = v[16]; v[8] = fminf(a, b); v[16] = fmaxf(a, b); }
    { const float a = v[4], b = v[20]; v[4] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[12], b = v[28]; v[12] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[12], b = v[20]; v[12] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[4], b = v[8]; v[4] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[12], b = v[16]; v[12] = fminf(a, b); v[16] = fmaxf(a, b); }
    { const float a = v[20], b = v[24]; v[20] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[2], b = v[18]; v[2] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[10], b = v[26]; v[10] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[10], b = v[18]; v[10] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[6], b = v[22]; v[6] = fminf(a, b); v[22] = fmaxf(a, b); }
    v[14] = fminf(v[14], v[30]);
    { const float a = v[14], b = v[22]; v[14] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[6], b = v[10]; v[6] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[14], b = v[18]; v[14] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[22], b = v[26]; v[22] = fminf(a, b); v[26] = fmaxf(a, b); }
    { const float a = v[2], b = v[4]; v[2] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[6], b = v[8]; v[6] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[10], b = v[12]; v[10] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[14], b = v[16]; v[14] = fminf(a, b); v[16] = fmaxf(a, b); }
    { const float a = v[18], b = v[20]; v[18] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[22], b = v[24]; v[22] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[26], b = v[28]; v[26] = fminf(a, b); v[28] = fmaxf(a, b); }
    { const float a = v[1], b = v[17]; v[1] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[9], b = v[25]; v[9] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[9], b = v[17]; v[9] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[5], b = v[21]; v[5] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[13], b = v[29]; v[13] = fminf(a, b); v[29] = fmaxf(a, b); }
    { const float a = v[13], b = v[21]; v[13] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[5], b = v[9]; v[5] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[13], b = v[17]; v[13] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[21], b = v[25]; v[21] = fminf(a, b); v[25] = fmaxf(a, b); }
    { const float a = v[3], b = v[19]; v[3] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[11], b = v[27]; v[11] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[11], b = v[19]; v[11] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[7], b = v[23]; v[7] = fminf(a, b); v[23] = fmaxf(a, b); }
    v[15] = fminf(v[15], v[31]);
    { const float a = v[15], b = v[23]; v[15] = fminf(a, b); v[23] = fmaxf(a, b); }
    { const float a = v[7], b = v[11]; v[7] = fminf(a, b); v[11] = fmaxf(a, b); }
    { const float a = v[15], b = v[19]; v[15] = fminf(a, b); v[19] = fmaxf(a, b); }
    { const float a = v[23], b = v[27]; v[23] = fminf(a, b); v[27] = fmaxf(a, b); }
    { const float a = v[3], b = v[5]; v[3] = fminf(a, b); v[5] = fmaxf(a, b); }
    { const float a = v[7], b = v[9]; v[7] = fminf(a, b); v[9] = fmaxf(a, b); }
    { const float a = v[11], b = v[13]; v[11] = fminf(a, b); v[13] = fmaxf(a, b); }
    { const float a = v[15], b = v[17]; v[15] = fminf(a, b); v[17] = fmaxf(a, b); }
    { const float a = v[19], b = v[21]; v[19] = fminf(a, b); v[21] = fmaxf(a, b); }
    { const float a = v[23], b = v[25]; v[23] = fminf(a, b); v[25] = fmaxf(a, b); }
    v[27] = fminf(v[27], v[29]);
    { const float a = v[1], b = v[2]; v[1] = fminf(a, b); v[2] = fmaxf(a, b); }
    { const float a = v[3], b = v[4]; v[3] = fminf(a, b); v[4] = fmaxf(a, b); }
    { const float a = v[5], b = v[6]; v[5] = fminf(a, b); v[6] = fmaxf(a, b); }
    { const float a = v[7], b = v[8]; v[7] = fminf(a, b); v[8] = fmaxf(a, b); }
    { const float a = v[9], b = v[10]; v[9] = fminf(a, b); v[10] = fmaxf(a, b); }
    { const float a = v[11], b = v[12]; v[11] = fminf(a, b); v[12] = fmaxf(a, b); }
    { const float a = v[13], b = v[14]; v[13] = fminf(a, b); v[14] = fmaxf(a, b); }
    { const float a = v[15], b = v[16]; v[15] = fminf(a, b); v[16] = fmaxf(a, b); }
    { const float a = v[17], b = v[18]; v[17] = fminf(a, b); v[18] = fmaxf(a, b); }
    { const float a = v[19], b = v[20]; v[19] = fminf(a, b); v[20] = fmaxf(a, b); }
    { const float a = v[21], b = v[22]; v[21] = fminf(a, b); v[22] = fmaxf(a, b); }
    { const float a = v[23], b = v[24]; v[23] = fminf(a, b); v[24] = fmaxf(a, b); }
    { const float a = v[25], b = v[26]; v[25] = fminf(a, b); v[26] = fmaxf(a, b); }
    v[27] = fminf(v[27], v[28]);
    { const float a = v[32], b = v[33]; v[32] = fminf(a, b); v[33] = fmaxf(a, b); }
    { const float a = v[34], b = v[35]; v[34] = fminf(a, b); v[35] = fmaxf(a, b); }
    { const float a = v[32], b = v[34]; v[32] = fminf(a, b); v[34] = fmaxf(a, b); }
    { const float a = v[33], b = v[35]; v[33] = fminf(a, b); v[35] = fmaxf(a, b); }
    { const float a = v[33], b = v[34]; v[33] = fminf(a, b); v[34] = fmaxf(a, b); }
    { const float a = v[36], b = v[37]; v[36] = fminf(a, b); v[37] = fmaxf(a, b); }
    { const float a = v[38], b = v[39]; v[38] = fminf(a, b); v[39] = fmaxf(a, b); }
    { const float a = v[36], b = v[38]; v[36] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[37], b = v[39]; v[37] = fminf(a, b); v[39] = fmaxf(a, b); }
    { const float a = v[37], b = v[38]; v[37] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[32], b = v[36]; v[32] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[34], b = v[38]; v[34] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[34], b = v[36]; v[34] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[33], b = v[37]; v[33] = fminf(a, b); v[37] = fmaxf(a, b); }
    { const float a = v[35], b = v[39]; v[35] = fminf(a, b); v[39] = fmaxf(a, b); }
    { const float a = v[35], b = v[37]; v[35] = fminf(a, b); v[37] = fmaxf(a, b); }
    { const float a = v[33], b = v[34]; v[33] = fminf(a, b); v[34] = fmaxf(a, b); }
    { const float a = v[35], b = v[36]; v[35] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[37], b = v[38]; v[37] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[40], b = v[41]; v[40] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[42], b = v[43]; v[42] = fminf(a, b); v[43] = fmaxf(a, b); }
    { const float a = v[40], b = v[42]; v[40] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[41], b = v[43]; v[41] = fminf(a, b); v[43] = fmaxf(a, b); }
    { const float a = v[41], b = v[42]; v[41] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[44], b = v[45]; v[44] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[46], b = v[47]; v[46] = fminf(a, b); v[47] = fmaxf(a, b); }
    { const float a = v[44], b = v[46]; v[44] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[45], b = v[47]; v[45] = fminf(a, b); v[47] = fmaxf(a, b); }
    { const float a = v[45], b = v[46]; v[45] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[40], b = v[44]; v[40] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[42], b = v[46]; v[42] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[42], b = v[44]; v[42] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[41], b = v[45]; v[41] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[43], b = v[47]; v[43] = fminf(a, b); v[47] = fmaxf(a, b); }
    { const float a = v[43], b = v[45]; v[43] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[41], b = v[42]; v[41] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[43], b = v[44]; v[43] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[45], b = v[46]; v[45] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[32], b = v[40]; v[32] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[36], b = v[44]; v[36] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[36], b = v[40]; v[36] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[34], b = v[42]; v[34] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[38], b = v[46]; v[38] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[38], b = v[42]; v[38] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[34], b = v[36]; v[34] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[38], b = v[40]; v[38] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[42], b = v[44]; v[42] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[33], b = v[41]; v[33] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[37], b = v[45]; v[37] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[37], b = v[41]; v[37] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[35], b = v[43]; v[35] = fminf(a, b); v[43] = fmaxf(a, b); }
    { const float a = v[39], b = v[47]; v[39] = fminf(a, b); v[47] = fmaxf(a, b); }
    { const float a = v[39], b = v[43]; v[39] = fminf(a, b); v[43] = fmaxf(a, b); }
    { const float a = v[35], b = v[37]; v[35] = fminf(a, b); v[37] = fmaxf(a, b); }
    { const float a = v[39], b = v[41]; v[39] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[43], b = v[45]; v[43] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[33], b = v[34]; v[33] = fminf(a, b); v[34] = fmaxf(a, b); }
    { const float a = v[35], b = v[36]; v[35] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[37], b = v[38]; v[37] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[39], b = v[40]; v[39] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[41], b = v[42]; v[41] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[43], b = v[44]; v[43] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[45], b = v[46]; v[45] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[32], b = v[48]; v[32] = fminf(a, b); v[48] = fmaxf(a, b); }
    { const float a = v[40], b = v[48]; v[40] = fminf(a, b); v[48] = fmaxf(a, b); }
    { const float a = v[36], b = v[40]; v[36] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[44], b = v[48]; v[44] = fminf(a, b); v[48] = fmaxf(a, b); }
    { const float a = v[38], b = v[42]; v[38] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[34], b = v[36]; v[34] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[38], b = v[40]; v[38] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[42], b = v[44]; v[42] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[46], b = v[48]; v[46] = fminf(a, b); v[48] = fmaxf(a, b); }
    { const float a = v[37], b = v[41]; v[37] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[39], b = v[43]; v[39] = fminf(a, b); v[43] = fmaxf(a, b); }
    { const float a = v[35], b = v[37]; v[35] = fminf(a, b); v[37] = fmaxf(a, b); }
    { const float a = v[39], b = v[41]; v[39] = fminf(a, b); v[41] = fmaxf(a, b); }
    { const float a = v[43], b = v[45]; v[43] = fminf(a, b); v[45] = fmaxf(a, b); }
    { const float a = v[33], b = v[34]; v[33] = fminf(a, b); v[34] = fmaxf(a, b); }
    { const float a = v[35], b = v[36]; v[35] = fminf(a, b); v[36] = fmaxf(a, b); }
    { const float a = v[37], b = v[38]; v[37] = fminf(a, b); v[38] = fmaxf(a, b); }
    { const float a = v[39], b = v[40]; v[39] = fminf(a, b); v[40] = fmaxf(a, b); }
    { const float a = v[41], b = v[42]; v[41] = fminf(a, b); v[42] = fmaxf(a, b); }
    { const float a = v[43], b = v[44]; v[43] = fminf(a, b); v[44] = fmaxf(a, b); }
    { const float a = v[45], b = v[46]; v[45] = fminf(a, b); v[46] = fmaxf(a, b); }
    { const float a = v[47], b = v[48]; v[47] = fminf(a, b); v[48] = fmaxf(a, b); }
    v[32] = fmaxf(v[0], v[32]);
    v[16] = fminf(v[16], v[48]);
    v[32] = fmaxf(v[16], v[32]);
    v[40] = fmaxf(v[8], v[40]);
    v[24] = fminf(v[24], v[40]);
    v[24] = fminf(v[24], v[32]);
    v[36] = fmaxf(v[4], v[36]);
    v[20] = fminf(v[20], v[36]);
    v[12] = fminf(v[12], v[44]);
    v[20] = fmaxf(v[12], v[20]);
    v[24] = fmaxf(v[20], v[24]);
    v[34] = fmaxf(v[2], v[34]);
    v[34] = fmaxf(v[18], v[34]);
    v[42] = fmaxf(v[10], v[42]);
    v[26] = fminf(v[26], v[42]);
    v[26] = fminf(v[26], v[34]);
    v[38] = fmaxf(v[6], v[38]);
    v[22] = fminf(v[22], v[38]);
    v[14] = fminf(v[14], v[46]);
    v[22] = fmaxf(v[14], v[22]);
    v[22] = fminf(v[22], v[26]);
    v[24] = fmaxf(v[22], v[24]);
    v[33] = fmaxf(v[1], v[33]);
    v[33] = fmaxf(v[17], v[33]);
    v[41] = fmaxf(v[9], v[41]);
    v[25] = fminf(v[25], v[41]);
    v[25] = fminf(v[25], v[33]);
    v[37] = fmaxf(v[5], v[37]);
    v[21] = fminf(v[21], v[37]);
    v[13] = fminf(v[13], v[45]);
    v[21] = fmaxf(v[13], v[21]);
    v[25] = fmaxf(v[21], v[25]);
    v[35] = fmaxf(v[3], v[35]);
    v[35] = fmaxf(v[19], v[35]);
    v[43] = fmaxf(v[11], v[43]);
    v[27] = fminf(v[27], v[43]);
    v[27] = fminf(v[27], v[35]);
    v[39] = fmaxf(v[7], v[39]);
    v[23] = fminf(v[23], v[39]);
    v[15] = fminf(v[15], v[47]);
    v[23] = fmaxf(v[15], v[23]);
    v[23] = fminf(v[23], v[27]);
    v[23] = fminf(v[23], v[25]);
    v[24] = fmaxf(v[23], v[24]);
    return v[24];
}

}  // namespace gp
