// GENERATED by paper_2211_14056_gb300/gen_tables.py -- do not edit.
// Heavy-quark pair + n gluons: colour matrices, sub-current tables and the
// straight-line quark-line code of one helicity lane (see the generator's
// docstring for the recursion it encodes).
#pragma once
#include "mf_device.cuh"
namespace mf {
template <int NG> struct TTNG;
template <int NG, int K> __device__ __forceinline__ const uint16_t* o3_table();
template <int NG, int K> __device__ __forceinline__ const uint16_t* o4_table();
template <int NG> __device__ __forceinline__ const uint8_t* blk_mask();
template <int NG> __device__ __forceinline__ const uint16_t* blk_off();
template <int NG> struct Paths;
template <int NG> struct ColourTC;
template <int NG> struct ColourPerm;
template <int NG> __device__ __forceinline__ const float* colour_frag_a();
template <int NG> __device__ __forceinline__ const int* colour_num_dev();
template <typename T> __device__ __forceinline__ V4<T> neg(const V4<T>& a) {
  V4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = -a.c[k];
  return o;
}
// colour matrix, 2 gluons: C = M / 3; orderings lexicographic
static constexpr int kColourDen2 = 3;
static const int kColourNum2[4] = {16, -2, -2, 16};
static __constant__ int kColourNumD2[4] = {16, -2, -2, 16};
template <> __device__ __forceinline__ const int* colour_num_dev<2>() { return kColourNumD2; }
// ---- 2 gluons: 3 blocks, 8 stored currents ----
template <> struct TTNG<2> {
  static constexpr int NBLK = 3;
  static constexpr int NSTORE = 8;
  static constexpr int NPERM = 2;
  static constexpr int FIRST[4] = {0, 0, 2, 3};
};
static __constant__ uint8_t kBlkMask2[3] = {1, 2, 3};
static __constant__ uint16_t kBlkOff2[3] = {0, 2, 4};
template <> __device__ __forceinline__ const uint8_t* blk_mask<2>() { return kBlkMask2; }
template <> __device__ __forceinline__ const uint16_t* blk_off<2>() { return kBlkOff2; }
static __constant__ uint16_t kO3_2_2[2] = {512, 1026};
template <> __device__ __forceinline__ const uint16_t* o3_table<2, 2>() { return kO3_2_2; }
static __constant__ uint8_t kPathMask2_1[2] = {1, 2};
static __constant__ uint16_t kPathBlk2_1[2] = {512, 1026};
static __constant__ uint8_t kPathFirst2_1[1] = {0};
static __constant__ uint8_t kFinalSigma2[2] = {1, 0};
static __constant__ uint16_t kFinalBlk2[4] = {1026, 9732, 512, 1540};
template <> struct Paths<2> {
  static __device__ __forceinline__ const uint8_t* mask_1() { return kPathMask2_1; }
  template <int LV> static __device__ __forceinline__ uint8_t mask(int p) {
    if constexpr (LV == 1) return kPathMask2_1[p];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ uint16_t blk(int p, int m) {
    if constexpr (LV == 1) return kPathBlk2_1[p * 1 + m];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ int first(int parent) {
    if constexpr (LV == 1) return kPathFirst2_1[parent];
    return 0;
  }
  static __device__ __forceinline__ uint8_t final_sigma(int p) { return kFinalSigma2[p]; }
  static __device__ __forceinline__ uint16_t final_blk(int p, int m) { return kFinalBlk2[p * 2 + m]; }
};
// J^dagger (D C) J of one helicity over the 2 colour orderings (D = 3).
template <typename T>
__device__ __forceinline__ T colour_form_2(const cplx<T> (&J)[2]) {
  T s = T(0);
  { cplx<T> y = T(8.0) * J[0];
    y = rfma(T(-2.0), J[1], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(8.0) * J[1];
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  return T(2) * s;
}
template <typename T> __device__ __forceinline__ T colour_form(const cplx<T> (&J)[2]) { return colour_form_2<T>(J); }
// D C as TF32 A fragments of mma.m16n8k8: [m-tile][k-step][register][lane]
template <> struct ColourTC<2> { static constexpr int MT = 1, KS = 1; };
static __device__ const float kColourFragA2[128] = {16.f, -2.f, 0.f, 0.f, -2.f, 16.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
template <> __device__ __forceinline__ const float* colour_frag_a<2>() { return kColourFragA2; }
// Half of J^dagger (D C) J / 2 for 2 orderings by the gluon relabelling
// symmetry (gen_tables.colour_orbit_terms): F(J) + F(J o perm) = J^dagger (D C) J / 2.
static __constant__ uint8_t kColourPerm2[2] = {1, 0};
template <typename T>
__device__ __forceinline__ T colour_form_orbit_2(const cplx<T> (&J)[2]) {
  T s = T(0);
  { cplx<T> y = T(8.0) * J[0];
    y = rfma(T(-1.0), J[1], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  return s;
}
template <typename T> __device__ __forceinline__ T colour_form_orbit(const cplx<T> (&J)[2]) { return colour_form_orbit_2<T>(J); }
template <> struct ColourPerm<2> {
  static __device__ __forceinline__ int at(int a) { return kColourPerm2[a]; }
};
// colour matrix, 3 gluons: C = M / 9; orderings lexicographic
static constexpr int kColourDen3 = 9;
static const int kColourNum3[36] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64};
static __constant__ int kColourNumD3[36] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64};
template <> __device__ __forceinline__ const int* colour_num_dev<3>() { return kColourNumD3; }
// ---- 3 gluons: 9 blocks, 42 stored currents ----
template <> struct TTNG<3> {
  static constexpr int NBLK = 9;
  static constexpr int NSTORE = 42;
  static constexpr int NPERM = 6;
  static constexpr int FIRST[5] = {0, 0, 3, 6, 9};
};
static __constant__ uint8_t kBlkMask3[9] = {1, 2, 4, 3, 5, 6, 7, 7, 7};
static __constant__ uint16_t kBlkOff3[9] = {0, 2, 4, 6, 10, 14, 18, 26, 34};
template <> __device__ __forceinline__ const uint8_t* blk_mask<3>() { return kBlkMask3; }
template <> __device__ __forceinline__ const uint16_t* blk_off<3>() { return kBlkOff3; }
static __constant__ uint16_t kO3_3_2[6] = {512, 1026, 512, 2052, 1026, 2052};
template <> __device__ __forceinline__ const uint16_t* o3_table<3, 2>() { return kO3_3_2; }
static __constant__ uint16_t kO3_3_3[12] = {512, 3086, 1542, 2052, 512, 11278, 2570, 1026, 1026, 2570, 9734, 2052};
template <> __device__ __forceinline__ const uint16_t* o3_table<3, 3>() { return kO3_3_3; }
static __constant__ uint16_t kO4_3_3[9] = {512, 1026, 2052, 512, 2052, 1026, 1026, 512, 2052};
template <> __device__ __forceinline__ const uint16_t* o4_table<3, 3>() { return kO4_3_3; }
static __constant__ uint8_t kPathMask3_1[3] = {1, 2, 4};
static __constant__ uint16_t kPathBlk3_1[3] = {512, 1026, 2052};
static __constant__ uint8_t kPathFirst3_1[1] = {0};
static __constant__ uint8_t kPathMask3_2[6] = {3, 5, 3, 6, 5, 6};
static __constant__ uint16_t kPathBlk3_2[12] = {1026, 9734, 2052, 10762, 512, 1542, 2052, 11278, 512, 2570, 1026, 3086};
static __constant__ uint8_t kPathFirst3_2[3] = {0, 2, 4};
static __constant__ uint8_t kFinalSigma3[6] = {5, 3, 4, 1, 2, 0};
static __constant__ uint16_t kFinalBlk3[18] = {2052, 11278, 3602, 1026, 3086, 3610, 2052, 10762, 3618, 512, 2570, 3610, 1026, 9734, 3618, 512, 1542, 3602};
template <> struct Paths<3> {
  static __device__ __forceinline__ const uint8_t* mask_1() { return kPathMask3_1; }
  static __device__ __forceinline__ const uint8_t* mask_2() { return kPathMask3_2; }
  template <int LV> static __device__ __forceinline__ uint8_t mask(int p) {
    if constexpr (LV == 1) return kPathMask3_1[p];
    if constexpr (LV == 2) return kPathMask3_2[p];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ uint16_t blk(int p, int m) {
    if constexpr (LV == 1) return kPathBlk3_1[p * 1 + m];
    if constexpr (LV == 2) return kPathBlk3_2[p * 2 + m];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ int first(int parent) {
    if constexpr (LV == 1) return kPathFirst3_1[parent];
    if constexpr (LV == 2) return kPathFirst3_2[parent];
    return 0;
  }
  static __device__ __forceinline__ uint8_t final_sigma(int p) { return kFinalSigma3[p]; }
  static __device__ __forceinline__ uint16_t final_blk(int p, int m) { return kFinalBlk3[p * 3 + m]; }
};
// J^dagger (D C) J of one helicity over the 6 colour orderings (D = 9).
template <typename T>
__device__ __forceinline__ T colour_form_3(const cplx<T> (&J)[6]) {
  T s = T(0);
  { cplx<T> y = T(32.0) * J[0];
    y = rfma(T(-8.0), J[1], y);
    y = rfma(T(-8.0), J[2], y);
    y = rfma(T(1.0), J[3], y);
    y = rfma(T(1.0), J[4], y);
    y = rfma(T(10.0), J[5], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[1];
    y = rfma(T(1.0), J[2], y);
    y = rfma(T(10.0), J[3], y);
    y = rfma(T(-8.0), J[4], y);
    y = rfma(T(1.0), J[5], y);
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[2];
    y = rfma(T(-8.0), J[3], y);
    y = rfma(T(10.0), J[4], y);
    y = rfma(T(1.0), J[5], y);
    s = fma(J[2].r, y.r, fma(J[2].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[3];
    y = rfma(T(1.0), J[4], y);
    y = rfma(T(-8.0), J[5], y);
    s = fma(J[3].r, y.r, fma(J[3].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[4];
    y = rfma(T(-8.0), J[5], y);
    s = fma(J[4].r, y.r, fma(J[4].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[5];
    s = fma(J[5].r, y.r, fma(J[5].i, y.i, s)); }
  return T(2) * s;
}
template <typename T> __device__ __forceinline__ T colour_form(const cplx<T> (&J)[6]) { return colour_form_3<T>(J); }
// D C as TF32 A fragments of mma.m16n8k8: [m-tile][k-step][register][lane]
template <> struct ColourTC<3> { static constexpr int MT = 1, KS = 1; };
static __device__ const float kColourFragA3[128] = {64.f, -8.f, -8.f, 1.f, -8.f, 64.f, 1.f, 10.f, -8.f, 1.f, 64.f, -8.f, 1.f, 10.f, -8.f, 64.f, 1.f, -8.f, 10.f, 1.f, 10.f, 1.f, 1.f, -8.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 10.f, 0.f, 0.f, -8.f, 1.f, 0.f, 0.f, 10.f, 1.f, 0.f, 0.f, 1.f, -8.f, 0.f, 0.f, 64.f, -8.f, 0.f, 0.f, -8.f, 64.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
template <> __device__ __forceinline__ const float* colour_frag_a<3>() { return kColourFragA3; }
// Half of J^dagger (D C) J / 2 for 6 orderings by the gluon relabelling
// symmetry (gen_tables.colour_orbit_terms): F(J) + F(J o perm) = J^dagger (D C) J / 2.
static __constant__ uint8_t kColourPerm3[6] = {2, 3, 0, 1, 5, 4};
template <typename T>
__device__ __forceinline__ T colour_form_orbit_3(const cplx<T> (&J)[6]) {
  T s = T(0);
  { cplx<T> y = T(32.0) * J[0];
    y = rfma(T(-8.0), J[1], y);
    y = rfma(T(-4.0), J[2], y);
    y = rfma(T(1.0), J[3], y);
    y = rfma(T(1.0), J[4], y);
    y = rfma(T(10.0), J[5], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[1];
    y = rfma(T(5.0), J[3], y);
    y = rfma(T(-8.0), J[4], y);
    y = rfma(T(1.0), J[5], y);
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  { cplx<T> y = T(32.0) * J[4];
    y = rfma(T(-4.0), J[5], y);
    s = fma(J[4].r, y.r, fma(J[4].i, y.i, s)); }
  return s;
}
template <typename T> __device__ __forceinline__ T colour_form_orbit(const cplx<T> (&J)[6]) { return colour_form_orbit_3<T>(J); }
template <> struct ColourPerm<3> {
  static __device__ __forceinline__ int at(int a) { return kColourPerm3[a]; }
};
// colour matrix, 4 gluons: C = M / 54; orderings lexicographic
static constexpr int kColourDen4 = 54;
static const int kColourNum4[576] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};
static __constant__ int kColourNumD4[576] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};
template <> __device__ __forceinline__ const int* colour_num_dev<4>() { return kColourNumD4; }
// ---- 4 gluons: 34 blocks, 320 stored currents ----
template <> struct TTNG<4> {
  static constexpr int NBLK = 34;
  static constexpr int NSTORE = 320;
  static constexpr int NPERM = 24;
  static constexpr int FIRST[6] = {0, 0, 4, 10, 22, 34};
};
static __constant__ uint8_t kBlkMask4[34] = {1, 2, 4, 8, 3, 5, 9, 6, 10, 12, 7, 11, 7, 13, 11, 13, 7, 11, 14, 14, 13, 14, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15};
static __constant__ uint16_t kBlkOff4[34] = {0, 2, 4, 6, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64, 72, 80, 88, 96, 104, 112, 120, 128, 144, 160, 176, 192, 208, 224, 240, 256, 272, 288, 304};
template <> __device__ __forceinline__ const uint8_t* blk_mask<4>() { return kBlkMask4; }
template <> __device__ __forceinline__ const uint16_t* blk_off<4>() { return kBlkOff4; }
static __constant__ uint16_t kO3_4_2[12] = {512, 1026, 512, 2052, 512, 4102, 1026, 2052, 1026, 4102, 2052, 4102};
template <> __device__ __forceinline__ const uint16_t* o3_table<4, 2>() { return kO3_4_2; }
static __constant__ uint16_t kO3_4_3[48] = {512, 3092, 1544, 2052, 512, 5144, 1544, 4102, 512, 11284, 2572, 1026, 512, 6172, 2572, 4102, 512, 13336, 4624, 1026, 512, 14364, 4624, 2052, 1026, 2572, 9736, 2052, 1026, 4624, 9736, 4102, 1026, 6172, 3092, 4102, 1026, 14364, 5144, 2052, 2052, 4624, 10764, 4102, 2052, 5144, 11284, 4102};
template <> __device__ __forceinline__ const uint16_t* o3_table<4, 3>() { return kO3_4_3; }
static __constant__ uint16_t kO4_4_3[36] = {512, 1026, 2052, 512, 1026, 4102, 512, 2052, 1026, 512, 2052, 4102, 512, 4102, 1026, 512, 4102, 2052, 1026, 512, 2052, 1026, 512, 4102, 1026, 2052, 4102, 1026, 4102, 2052, 2052, 512, 4102, 2052, 1026, 4102};
template <> __device__ __forceinline__ const uint16_t* o4_table<4, 3>() { return kO4_4_3; }
static __constant__ uint16_t kO3_4_4[72] = {512, 7264, 1544, 6172, 3616, 4102, 512, 7272, 1544, 14364, 5672, 2052, 512, 7288, 2572, 5144, 3632, 4102, 512, 7272, 2572, 13336, 6712, 1026, 512, 7288, 4624, 3092, 5696, 2052, 512, 7264, 4624, 11284, 6728, 1026, 1026, 6712, 9736, 6172, 3664, 4102, 1026, 6728, 9736, 14364, 5720, 2052, 1026, 6768, 3092, 4624, 3632, 4102, 1026, 6768, 5144, 2572, 5696, 2052, 2052, 5672, 10764, 5144, 3664, 4102, 2052, 5720, 11284, 4624, 3616, 4102};
template <> __device__ __forceinline__ const uint16_t* o3_table<4, 4>() { return kO3_4_4; }
static __constant__ uint16_t kO4_4_4[108] = {512, 1026, 6172, 512, 3092, 4102, 1544, 2052, 4102, 512, 1026, 14364, 512, 5144, 2052, 1544, 4102, 2052, 512, 2052, 5144, 512, 11284, 4102, 2572, 1026, 4102, 512, 2052, 13336, 512, 6172, 1026, 2572, 4102, 1026, 512, 4102, 3092, 512, 13336, 2052, 4624, 1026, 2052, 512, 4102, 11284, 512, 14364, 1026, 4624, 2052, 1026, 1026, 512, 6172, 1026, 2572, 4102, 9736, 2052, 4102, 1026, 512, 14364, 1026, 4624, 2052, 9736, 4102, 2052, 1026, 2052, 4624, 1026, 10764, 4102, 3092, 512, 4102, 1026, 4102, 2572, 1026, 12816, 2052, 5144, 512, 2052, 2052, 512, 5144, 2052, 1544, 4102, 10764, 1026, 4102, 2052, 1026, 4624, 2052, 9736, 4102, 11284, 512, 4102};
template <> __device__ __forceinline__ const uint16_t* o4_table<4, 4>() { return kO4_4_4; }
static __constant__ uint8_t kPathMask4_1[4] = {1, 2, 4, 8};
static __constant__ uint16_t kPathBlk4_1[4] = {512, 1026, 2052, 4102};
static __constant__ uint8_t kPathFirst4_1[1] = {0};
static __constant__ uint8_t kPathMask4_2[12] = {3, 5, 9, 3, 6, 10, 5, 6, 12, 9, 10, 12};
static __constant__ uint16_t kPathBlk4_2[24] = {1026, 9736, 2052, 10764, 4102, 12816, 512, 1544, 2052, 11284, 4102, 13336, 512, 2572, 1026, 3092, 4102, 14364, 512, 4624, 1026, 5144, 2052, 6172};
static __constant__ uint8_t kPathFirst4_2[4] = {0, 3, 6, 9};
static __constant__ uint8_t kPathMask4_3[24] = {7, 11, 7, 13, 11, 13, 7, 11, 7, 14, 11, 14, 7, 13, 7, 14, 13, 14, 11, 13, 11, 14, 13, 14};
static __constant__ uint16_t kPathBlk4_3[72] = {2052, 11284, 3616, 4102, 13336, 5672, 1026, 3092, 3632, 4102, 14364, 6712, 1026, 5144, 5696, 2052, 6172, 6728, 2052, 10764, 3664, 4102, 12816, 5720, 512, 2572, 3632, 4102, 14364, 7264, 512, 4624, 5696, 2052, 6172, 7272, 1026, 9736, 3664, 4102, 12816, 6768, 512, 1544, 3616, 4102, 13336, 7288, 512, 4624, 6728, 1026, 5144, 7272, 1026, 9736, 5720, 2052, 10764, 6768, 512, 1544, 5672, 2052, 11284, 7288, 512, 2572, 6712, 1026, 3092, 7264};
static __constant__ uint8_t kPathFirst4_3[12] = {0, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22};
static __constant__ uint8_t kL3Pair4[24] = {3, 5, 1, 4, 0, 2, 9, 11, 7, 10, 6, 8, 15, 17, 13, 16, 12, 14, 21, 23, 19, 22, 18, 20};
static __constant__ uint8_t kL3Miss4[12] = {1, 2, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2};
static __constant__ uint8_t kFinalSigma4[24] = {23, 17, 21, 11, 15, 9, 22, 16, 19, 5, 13, 3, 20, 10, 18, 4, 7, 1, 14, 8, 12, 2, 6, 0};
static __constant__ uint16_t kFinalBlk4[96] = {4102, 14364, 7264, 16000, 2052, 6172, 7272, 16016, 4102, 13336, 7288, 16032, 1026, 5144, 7272, 16048, 2052, 11284, 7288, 16064, 1026, 3092, 7264, 16080, 4102, 14364, 6712, 16096, 2052, 6172, 6728, 16112, 4102, 12816, 6768, 16128, 512, 4624, 6728, 7888, 2052, 10764, 6768, 16144, 512, 2572, 6712, 7856, 4102, 13336, 5672, 16160, 1026, 5144, 5696, 7952, 4102, 12816, 5720, 16176, 512, 4624, 5696, 7872, 1026, 9736, 5720, 7920, 512, 1544, 5672, 7824, 2052, 11284, 3616, 7984, 1026, 3092, 3632, 7936, 2052, 10764, 3664, 7968, 512, 2572, 3632, 7840, 1026, 9736, 3664, 7904, 512, 1544, 3616, 7808};
template <> struct Paths<4> {
  static __device__ __forceinline__ const uint8_t* mask_1() { return kPathMask4_1; }
  static __device__ __forceinline__ const uint8_t* mask_2() { return kPathMask4_2; }
  static __device__ __forceinline__ const uint8_t* mask_3() { return kPathMask4_3; }
  template <int LV> static __device__ __forceinline__ uint8_t mask(int p) {
    if constexpr (LV == 1) return kPathMask4_1[p];
    if constexpr (LV == 2) return kPathMask4_2[p];
    if constexpr (LV == 3) return kPathMask4_3[p];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ uint16_t blk(int p, int m) {
    if constexpr (LV == 1) return kPathBlk4_1[p * 1 + m];
    if constexpr (LV == 2) return kPathBlk4_2[p * 2 + m];
    if constexpr (LV == 3) return kPathBlk4_3[p * 3 + m];
    return 0;
  }
  template <int LV> static __device__ __forceinline__ int first(int parent) {
    if constexpr (LV == 1) return kPathFirst4_1[parent];
    if constexpr (LV == 2) return kPathFirst4_2[parent];
    if constexpr (LV == 3) return kPathFirst4_3[parent];
    return 0;
  }
  static __device__ __forceinline__ uint8_t final_sigma(int p) { return kFinalSigma4[p]; }
  static __device__ __forceinline__ uint16_t final_blk(int p, int m) { return kFinalBlk4[p * 4 + m]; }
};
// J^dagger (D C) J of one helicity over the 24 colour orderings (D = 54).
template <typename T>
__device__ __forceinline__ T colour_form_4(const cplx<T> (&J)[24]) {
  T s = T(0);
  { cplx<T> y = T(256.0) * J[0];
    y = rfma(T(-64.0), J[1], y);
    y = rfma(T(-64.0), J[2], y);
    y = rfma(T(8.0), J[3], y);
    y = rfma(T(8.0), J[4], y);
    y = rfma(T(80.0), J[5], y);
    y = rfma(T(-64.0), J[6], y);
    y = rfma(T(8.0), J[7], y);
    y = rfma(T(8.0), J[8], y);
    y = rfma(T(-1.0), J[9], y);
    y = rfma(T(-1.0), J[10], y);
    y = rfma(T(-10.0), J[11], y);
    y = rfma(T(8.0), J[12], y);
    y = rfma(T(-1.0), J[13], y);
    y = rfma(T(80.0), J[14], y);
    y = rfma(T(-10.0), J[15], y);
    y = rfma(T(71.0), J[16], y);
    y = rfma(T(62.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(-10.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(62.0), J[22], y);
    y = rfma(T(-28.0), J[23], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[1];
    y = rfma(T(8.0), J[2], y);
    y = rfma(T(80.0), J[3], y);
    y = rfma(T(-64.0), J[4], y);
    y = rfma(T(8.0), J[5], y);
    y = rfma(T(8.0), J[6], y);
    y = rfma(T(-64.0), J[7], y);
    y = rfma(T(-1.0), J[8], y);
    y = rfma(T(-10.0), J[9], y);
    y = rfma(T(8.0), J[10], y);
    y = rfma(T(-1.0), J[11], y);
    y = rfma(T(-1.0), J[12], y);
    y = rfma(T(-10.0), J[13], y);
    y = rfma(T(-10.0), J[14], y);
    y = rfma(T(62.0), J[15], y);
    y = rfma(T(62.0), J[16], y);
    y = rfma(T(-28.0), J[17], y);
    y = rfma(T(8.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(80.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(71.0), J[22], y);
    y = rfma(T(62.0), J[23], y);
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[2];
    y = rfma(T(-64.0), J[3], y);
    y = rfma(T(80.0), J[4], y);
    y = rfma(T(8.0), J[5], y);
    y = rfma(T(8.0), J[6], y);
    y = rfma(T(-1.0), J[7], y);
    y = rfma(T(80.0), J[8], y);
    y = rfma(T(-10.0), J[9], y);
    y = rfma(T(71.0), J[10], y);
    y = rfma(T(62.0), J[11], y);
    y = rfma(T(-64.0), J[12], y);
    y = rfma(T(8.0), J[13], y);
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(-1.0), J[15], y);
    y = rfma(T(-1.0), J[16], y);
    y = rfma(T(-10.0), J[17], y);
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(62.0), J[20], y);
    y = rfma(T(-28.0), J[21], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(62.0), J[23], y);
    s = fma(J[2].r, y.r, fma(J[2].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[3];
    y = rfma(T(8.0), J[4], y);
    y = rfma(T(-64.0), J[5], y);
    y = rfma(T(-1.0), J[6], y);
    y = rfma(T(-10.0), J[7], y);
    y = rfma(T(-10.0), J[8], y);
    y = rfma(T(62.0), J[9], y);
    y = rfma(T(62.0), J[10], y);
    y = rfma(T(-28.0), J[11], y);
    y = rfma(T(8.0), J[12], y);
    y = rfma(T(-64.0), J[13], y);
    y = rfma(T(-1.0), J[14], y);
    y = rfma(T(-10.0), J[15], y);
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(-1.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(8.0), J[19], y);
    y = rfma(T(71.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(80.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[3].r, y.r, fma(J[3].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[4];
    y = rfma(T(-64.0), J[5], y);
    y = rfma(T(-1.0), J[6], y);
    y = rfma(T(8.0), J[7], y);
    y = rfma(T(71.0), J[8], y);
    y = rfma(T(62.0), J[9], y);
    y = rfma(T(80.0), J[10], y);
    y = rfma(T(-10.0), J[11], y);
    y = rfma(T(-10.0), J[12], y);
    y = rfma(T(-1.0), J[13], y);
    y = rfma(T(62.0), J[14], y);
    y = rfma(T(-28.0), J[15], y);
    y = rfma(T(-10.0), J[16], y);
    y = rfma(T(62.0), J[17], y);
    y = rfma(T(-64.0), J[18], y);
    y = rfma(T(8.0), J[19], y);
    y = rfma(T(8.0), J[20], y);
    y = rfma(T(-1.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[4].r, y.r, fma(J[4].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[5];
    y = rfma(T(-10.0), J[6], y);
    y = rfma(T(-1.0), J[7], y);
    y = rfma(T(62.0), J[8], y);
    y = rfma(T(-28.0), J[9], y);
    y = rfma(T(-10.0), J[10], y);
    y = rfma(T(62.0), J[11], y);
    y = rfma(T(-1.0), J[12], y);
    y = rfma(T(8.0), J[13], y);
    y = rfma(T(71.0), J[14], y);
    y = rfma(T(62.0), J[15], y);
    y = rfma(T(80.0), J[16], y);
    y = rfma(T(-10.0), J[17], y);
    y = rfma(T(8.0), J[18], y);
    y = rfma(T(-64.0), J[19], y);
    y = rfma(T(-1.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[5].r, y.r, fma(J[5].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[6];
    y = rfma(T(-64.0), J[7], y);
    y = rfma(T(-64.0), J[8], y);
    y = rfma(T(8.0), J[9], y);
    y = rfma(T(8.0), J[10], y);
    y = rfma(T(80.0), J[11], y);
    y = rfma(T(80.0), J[12], y);
    y = rfma(T(-10.0), J[13], y);
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(-1.0), J[15], y);
    y = rfma(T(62.0), J[16], y);
    y = rfma(T(71.0), J[17], y);
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(62.0), J[19], y);
    y = rfma(T(-1.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(-28.0), J[22], y);
    y = rfma(T(62.0), J[23], y);
    s = fma(J[6].r, y.r, fma(J[6].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[7];
    y = rfma(T(8.0), J[8], y);
    y = rfma(T(80.0), J[9], y);
    y = rfma(T(-64.0), J[10], y);
    y = rfma(T(8.0), J[11], y);
    y = rfma(T(-10.0), J[12], y);
    y = rfma(T(62.0), J[13], y);
    y = rfma(T(-1.0), J[14], y);
    y = rfma(T(-10.0), J[15], y);
    y = rfma(T(-28.0), J[16], y);
    y = rfma(T(62.0), J[17], y);
    y = rfma(T(80.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(8.0), J[20], y);
    y = rfma(T(-1.0), J[21], y);
    y = rfma(T(62.0), J[22], y);
    y = rfma(T(71.0), J[23], y);
    s = fma(J[7].r, y.r, fma(J[7].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[8];
    y = rfma(T(-64.0), J[9], y);
    y = rfma(T(80.0), J[10], y);
    y = rfma(T(8.0), J[11], y);
    y = rfma(T(8.0), J[12], y);
    y = rfma(T(-1.0), J[13], y);
    y = rfma(T(-64.0), J[14], y);
    y = rfma(T(8.0), J[15], y);
    y = rfma(T(-10.0), J[16], y);
    y = rfma(T(-1.0), J[17], y);
    y = rfma(T(62.0), J[18], y);
    y = rfma(T(-28.0), J[19], y);
    y = rfma(T(-10.0), J[20], y);
    y = rfma(T(-1.0), J[21], y);
    y = rfma(T(62.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[8].r, y.r, fma(J[8].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[9];
    y = rfma(T(8.0), J[10], y);
    y = rfma(T(-64.0), J[11], y);
    y = rfma(T(-1.0), J[12], y);
    y = rfma(T(-10.0), J[13], y);
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(-64.0), J[15], y);
    y = rfma(T(-1.0), J[16], y);
    y = rfma(T(8.0), J[17], y);
    y = rfma(T(71.0), J[18], y);
    y = rfma(T(62.0), J[19], y);
    y = rfma(T(-1.0), J[20], y);
    y = rfma(T(8.0), J[21], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(80.0), J[23], y);
    s = fma(J[9].r, y.r, fma(J[9].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[10];
    y = rfma(T(-64.0), J[11], y);
    y = rfma(T(62.0), J[12], y);
    y = rfma(T(-28.0), J[13], y);
    y = rfma(T(-10.0), J[14], y);
    y = rfma(T(-1.0), J[15], y);
    y = rfma(T(62.0), J[16], y);
    y = rfma(T(-10.0), J[17], y);
    y = rfma(T(8.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(-64.0), J[20], y);
    y = rfma(T(8.0), J[21], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[10].r, y.r, fma(J[10].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[11];
    y = rfma(T(71.0), J[12], y);
    y = rfma(T(62.0), J[13], y);
    y = rfma(T(-1.0), J[14], y);
    y = rfma(T(8.0), J[15], y);
    y = rfma(T(-10.0), J[16], y);
    y = rfma(T(80.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(8.0), J[20], y);
    y = rfma(T(-64.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[11].r, y.r, fma(J[11].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[12];
    y = rfma(T(-64.0), J[13], y);
    y = rfma(T(-64.0), J[14], y);
    y = rfma(T(8.0), J[15], y);
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(80.0), J[17], y);
    y = rfma(T(62.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(-28.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[12].r, y.r, fma(J[12].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[13];
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(80.0), J[15], y);
    y = rfma(T(-64.0), J[16], y);
    y = rfma(T(8.0), J[17], y);
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(80.0), J[19], y);
    y = rfma(T(62.0), J[20], y);
    y = rfma(T(71.0), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[13].r, y.r, fma(J[13].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[14];
    y = rfma(T(-64.0), J[15], y);
    y = rfma(T(80.0), J[16], y);
    y = rfma(T(8.0), J[17], y);
    y = rfma(T(-28.0), J[18], y);
    y = rfma(T(62.0), J[19], y);
    y = rfma(T(62.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[14].r, y.r, fma(J[14].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[15];
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(-64.0), J[17], y);
    y = rfma(T(62.0), J[18], y);
    y = rfma(T(71.0), J[19], y);
    y = rfma(T(-10.0), J[20], y);
    y = rfma(T(80.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[15].r, y.r, fma(J[15].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[16];
    y = rfma(T(-64.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(8.0), J[19], y);
    y = rfma(T(-10.0), J[20], y);
    y = rfma(T(-1.0), J[21], y);
    y = rfma(T(-64.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[16].r, y.r, fma(J[16].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[17];
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(-1.0), J[20], y);
    y = rfma(T(8.0), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-64.0), J[23], y);
    s = fma(J[17].r, y.r, fma(J[17].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[18];
    y = rfma(T(-64.0), J[19], y);
    y = rfma(T(-64.0), J[20], y);
    y = rfma(T(8.0), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(80.0), J[23], y);
    s = fma(J[18].r, y.r, fma(J[18].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[19];
    y = rfma(T(8.0), J[20], y);
    y = rfma(T(80.0), J[21], y);
    y = rfma(T(-64.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[19].r, y.r, fma(J[19].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[20];
    y = rfma(T(-64.0), J[21], y);
    y = rfma(T(80.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[20].r, y.r, fma(J[20].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[21];
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-64.0), J[23], y);
    s = fma(J[21].r, y.r, fma(J[21].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[22];
    y = rfma(T(-64.0), J[23], y);
    s = fma(J[22].r, y.r, fma(J[22].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[23];
    s = fma(J[23].r, y.r, fma(J[23].i, y.i, s)); }
  return T(2) * s;
}
template <typename T> __device__ __forceinline__ T colour_form(const cplx<T> (&J)[24]) { return colour_form_4<T>(J); }
// D C as TF32 A fragments of mma.m16n8k8: [m-tile][k-step][register][lane]
template <> struct ColourTC<4> { static constexpr int MT = 2, KS = 3; };
static __device__ const float kColourFragA4[768] = {512.f, -64.f, -64.f, 8.f, -64.f, 512.f, 8.f, 80.f, -64.f, 8.f, 512.f, -64.f, 8.f, 80.f, -64.f, 512.f, 8.f, -64.f, 80.f, 8.f, 80.f, 8.f, 8.f, -64.f, -64.f, 8.f, 8.f, -1.f, 8.f, -64.f, -1.f, -10.f, 8.f, -1.f, 80.f, -10.f, -1.f, -10.f, -10.f, 62.f, -1.f, 8.f, 71.f, 62.f, -10.f, -1.f, 62.f, -28.f, 8.f, -1.f, -64.f, 8.f, -1.f, -10.f, 8.f, -64.f, 80.f, -10.f, 8.f, -1.f, -10.f, 62.f, -1.f, -10.f, 8.f, 80.f, -64.f, 8.f, -64.f, 8.f, 8.f, -64.f, 80.f, 8.f, 8.f, -1.f, 8.f, -64.f, -1.f, -10.f, 512.f, -64.f, -1.f, 8.f, -64.f, 512.f, -10.f, -1.f, -1.f, -10.f, 512.f, -64.f, 8.f, -1.f, -64.f, 512.f, 71.f, 62.f, -64.f, 8.f, 62.f, -28.f, 8.f, 80.f, 80.f, -10.f, 8.f, -64.f, -10.f, 62.f, 80.f, 8.f, -10.f, -1.f, 80.f, -10.f, -1.f, 8.f, -10.f, 62.f, 62.f, 71.f, 8.f, -1.f, -28.f, 62.f, -1.f, -10.f, 8.f, -1.f, -1.f, -10.f, -1.f, -10.f, 8.f, -1.f, 80.f, -10.f, 71.f, 62.f, -10.f, 62.f, 62.f, -28.f, 71.f, 62.f, 80.f, -10.f, 62.f, -28.f, -10.f, 62.f, -64.f, 8.f, 8.f, 80.f, 8.f, 80.f, -64.f, 8.f, 512.f, -64.f, 80.f, 8.f, -64.f, 512.f, 8.f, -64.f, 80.f, 8.f, 512.f, -64.f, 8.f, -64.f, -64.f, 512.f, 8.f, -1.f, 62.f, 71.f, -1.f, -10.f, -28.f, 62.f, -64.f, 8.f, -10.f, -1.f, 8.f, -64.f, -1.f, 8.f, 8.f, -1.f, 80.f, -10.f, -1.f, -10.f, -10.f, 62.f, -64.f, 8.f, 8.f, -1.f, 8.f, -64.f, -1.f, -10.f, -10.f, -1.f, 62.f, -28.f, -1.f, 8.f, 71.f, 62.f, 80.f, -10.f, 8.f, -1.f, -10.f, 62.f, -1.f, -10.f, 8.f, -1.f, -64.f, 8.f, -1.f, -10.f, 8.f, -64.f, 62.f, -28.f, -10.f, -1.f, 71.f, 62.f, -1.f, 8.f, 512.f, -64.f, -64.f, 8.f, -64.f, 512.f, 8.f, 80.f, -64.f, 8.f, 512.f, -64.f, 8.f, 80.f, -64.f, 512.f, 71.f, 62.f, -1.f, -10.f, 62.f, -28.f, 8.f, -1.f, -1.f, -10.f, -10.f, -1.f, 8.f, -1.f, -1.f, 8.f, -10.f, 62.f, -64.f, 8.f, 80.f, -10.f, 8.f, -64.f, 62.f, 71.f, -10.f, 62.f, -28.f, 62.f, 80.f, -10.f, -10.f, -1.f, 62.f, -28.f, -1.f, 8.f, 71.f, 62.f, 62.f, -10.f, 8.f, -1.f, -10.f, 80.f, -1.f, -10.f, 8.f, 80.f, 62.f, -10.f, -64.f, 8.f, -10.f, 80.f, 80.f, 8.f, -28.f, 62.f, 8.f, -64.f, 62.f, 71.f, -10.f, 62.f, 62.f, -28.f, 80.f, -10.f, 71.f, 62.f, 62.f, -28.f, -10.f, 62.f, 71.f, 62.f, 80.f, -10.f, 8.f, -1.f, -1.f, -10.f, -1.f, -10.f, 8.f, -1.f, -1.f, -10.f, -28.f, 62.f, 8.f, -1.f, 62.f, 71.f, -10.f, -1.f, 62.f, -10.f, -1.f, 8.f, -10.f, 80.f, -64.f, 8.f, -10.f, -1.f, 8.f, -64.f, -1.f, 8.f, -28.f, 62.f, -1.f, -10.f, 62.f, 71.f, 8.f, -1.f, 62.f, -10.f, -10.f, -1.f, -10.f, 80.f, -1.f, 8.f, 71.f, 62.f, -1.f, 8.f, 62.f, -28.f, -10.f, -1.f, -1.f, 8.f, -10.f, -1.f, -10.f, -1.f, -1.f, 8.f, -10.f, 80.f, 62.f, 71.f, 62.f, -10.f, -28.f, 62.f, 62.f, 71.f, -10.f, 80.f, -28.f, 62.f, 62.f, -10.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -10.f, 80.f, 62.f, -28.f, 62.f, -10.f, 71.f, 62.f, -64.f, 8.f, -10.f, 80.f, 8.f, -64.f, 62.f, -10.f, 8.f, -1.f, -1.f, 8.f, -1.f, -10.f, -10.f, -1.f, -1.f, 8.f, -28.f, 62.f, -10.f, -1.f, 62.f, 71.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -10.f, -1.f, 62.f, -10.f, -1.f, 8.f, -10.f, 80.f, 62.f, 71.f, 8.f, -1.f, -28.f, 62.f, -1.f, -10.f, -10.f, -1.f, -64.f, 8.f, -1.f, 8.f, 8.f, -64.f, 62.f, -10.f, -10.f, -1.f, -10.f, 80.f, -1.f, 8.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 8.f, -64.f, 80.f, 8.f, 80.f, 8.f, 8.f, -64.f, 62.f, -10.f, -28.f, 62.f, -10.f, 80.f, 62.f, 71.f, -28.f, 62.f, 62.f, -10.f, 62.f, 71.f, -10.f, 80.f, -1.f, 8.f, -10.f, -1.f, -10.f, -1.f, -1.f, 8.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 512.f, -64.f, -1.f, 8.f, -64.f, 512.f, -10.f, -1.f, -1.f, -10.f, 512.f, -64.f, 8.f, -1.f, -64.f, 512.f, -10.f, -1.f, -64.f, 8.f, -1.f, 8.f, 8.f, 80.f, -64.f, 8.f, 8.f, -64.f, 8.f, -64.f, 80.f, 8.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -10.f, -1.f, -64.f, 8.f, -1.f, 8.f, 8.f, -64.f, -64.f, 8.f, 8.f, 80.f, 8.f, 80.f, -64.f, 8.f, 512.f, -64.f, 80.f, 8.f, -64.f, 512.f, 8.f, -64.f, 80.f, 8.f, 512.f, -64.f, 8.f, -64.f, -64.f, 512.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
template <> __device__ __forceinline__ const float* colour_frag_a<4>() { return kColourFragA4; }
// Half of J^dagger (D C) J / 2 for 24 orderings by the gluon relabelling
// symmetry (gen_tables.colour_orbit_terms): F(J) + F(J o perm) = J^dagger (D C) J / 2.
static __constant__ uint8_t kColourPerm4[24] = {7, 6, 10, 11, 8, 9, 1, 0, 4, 5, 2, 3, 20, 21, 18, 19, 23, 22, 14, 15, 12, 13, 17, 16};
template <typename T>
__device__ __forceinline__ T colour_form_orbit_4(const cplx<T> (&J)[24]) {
  T s = T(0);
  { cplx<T> y = T(256.0) * J[0];
    y = rfma(T(-64.0), J[1], y);
    y = rfma(T(-64.0), J[2], y);
    y = rfma(T(8.0), J[3], y);
    y = rfma(T(8.0), J[4], y);
    y = rfma(T(80.0), J[5], y);
    y = rfma(T(-64.0), J[6], y);
    y = rfma(T(4.0), J[7], y);
    y = rfma(T(8.0), J[8], y);
    y = rfma(T(-1.0), J[9], y);
    y = rfma(T(-1.0), J[10], y);
    y = rfma(T(-10.0), J[11], y);
    y = rfma(T(8.0), J[12], y);
    y = rfma(T(-1.0), J[13], y);
    y = rfma(T(80.0), J[14], y);
    y = rfma(T(-10.0), J[15], y);
    y = rfma(T(71.0), J[16], y);
    y = rfma(T(62.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(-10.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(62.0), J[22], y);
    y = rfma(T(-28.0), J[23], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[1];
    y = rfma(T(8.0), J[2], y);
    y = rfma(T(80.0), J[3], y);
    y = rfma(T(-64.0), J[4], y);
    y = rfma(T(8.0), J[5], y);
    y = rfma(T(4.0), J[6], y);
    y = rfma(T(-1.0), J[8], y);
    y = rfma(T(-10.0), J[9], y);
    y = rfma(T(8.0), J[10], y);
    y = rfma(T(-1.0), J[11], y);
    y = rfma(T(-1.0), J[12], y);
    y = rfma(T(-10.0), J[13], y);
    y = rfma(T(-10.0), J[14], y);
    y = rfma(T(62.0), J[15], y);
    y = rfma(T(62.0), J[16], y);
    y = rfma(T(-28.0), J[17], y);
    y = rfma(T(8.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(80.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(71.0), J[22], y);
    y = rfma(T(62.0), J[23], y);
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[2];
    y = rfma(T(-64.0), J[3], y);
    y = rfma(T(80.0), J[4], y);
    y = rfma(T(8.0), J[5], y);
    y = rfma(T(80.0), J[8], y);
    y = rfma(T(-10.0), J[9], y);
    y = rfma(T(35.5), J[10], y);
    y = rfma(T(62.0), J[11], y);
    y = rfma(T(-64.0), J[12], y);
    y = rfma(T(8.0), J[13], y);
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(-1.0), J[15], y);
    y = rfma(T(-1.0), J[16], y);
    y = rfma(T(-10.0), J[17], y);
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(-1.0), J[19], y);
    y = rfma(T(62.0), J[20], y);
    y = rfma(T(-28.0), J[21], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(62.0), J[23], y);
    s = fma(J[2].r, y.r, fma(J[2].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[3];
    y = rfma(T(8.0), J[4], y);
    y = rfma(T(-64.0), J[5], y);
    y = rfma(T(-10.0), J[8], y);
    y = rfma(T(62.0), J[9], y);
    y = rfma(T(-14.0), J[11], y);
    y = rfma(T(8.0), J[12], y);
    y = rfma(T(-64.0), J[13], y);
    y = rfma(T(-1.0), J[14], y);
    y = rfma(T(-10.0), J[15], y);
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(-1.0), J[17], y);
    y = rfma(T(-1.0), J[18], y);
    y = rfma(T(8.0), J[19], y);
    y = rfma(T(71.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(80.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[3].r, y.r, fma(J[3].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[4];
    y = rfma(T(-64.0), J[5], y);
    y = rfma(T(35.5), J[8], y);
    y = rfma(T(62.0), J[9], y);
    y = rfma(T(-10.0), J[12], y);
    y = rfma(T(-1.0), J[13], y);
    y = rfma(T(62.0), J[14], y);
    y = rfma(T(-28.0), J[15], y);
    y = rfma(T(-10.0), J[16], y);
    y = rfma(T(62.0), J[17], y);
    y = rfma(T(-64.0), J[18], y);
    y = rfma(T(8.0), J[19], y);
    y = rfma(T(8.0), J[20], y);
    y = rfma(T(-1.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[4].r, y.r, fma(J[4].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[5];
    y = rfma(T(-14.0), J[9], y);
    y = rfma(T(-1.0), J[12], y);
    y = rfma(T(8.0), J[13], y);
    y = rfma(T(71.0), J[14], y);
    y = rfma(T(62.0), J[15], y);
    y = rfma(T(80.0), J[16], y);
    y = rfma(T(-10.0), J[17], y);
    y = rfma(T(8.0), J[18], y);
    y = rfma(T(-64.0), J[19], y);
    y = rfma(T(-1.0), J[20], y);
    y = rfma(T(-10.0), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[5].r, y.r, fma(J[5].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[12];
    y = rfma(T(-64.0), J[13], y);
    y = rfma(T(-64.0), J[14], y);
    y = rfma(T(8.0), J[15], y);
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(80.0), J[17], y);
    y = rfma(T(62.0), J[18], y);
    y = rfma(T(-10.0), J[19], y);
    y = rfma(T(-14.0), J[20], y);
    y = rfma(T(62.0), J[21], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(-10.0), J[23], y);
    s = fma(J[12].r, y.r, fma(J[12].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[13];
    y = rfma(T(8.0), J[14], y);
    y = rfma(T(80.0), J[15], y);
    y = rfma(T(-64.0), J[16], y);
    y = rfma(T(8.0), J[17], y);
    y = rfma(T(-10.0), J[18], y);
    y = rfma(T(80.0), J[19], y);
    y = rfma(T(35.5), J[21], y);
    y = rfma(T(8.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[13].r, y.r, fma(J[13].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[14];
    y = rfma(T(-64.0), J[15], y);
    y = rfma(T(80.0), J[16], y);
    y = rfma(T(8.0), J[17], y);
    y = rfma(T(-14.0), J[18], y);
    y = rfma(T(62.0), J[19], y);
    y = rfma(T(-10.0), J[22], y);
    y = rfma(T(-1.0), J[23], y);
    s = fma(J[14].r, y.r, fma(J[14].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[15];
    y = rfma(T(8.0), J[16], y);
    y = rfma(T(-64.0), J[17], y);
    y = rfma(T(35.5), J[19], y);
    y = rfma(T(-1.0), J[22], y);
    y = rfma(T(8.0), J[23], y);
    s = fma(J[15].r, y.r, fma(J[15].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[16];
    y = rfma(T(-64.0), J[17], y);
    y = rfma(T(-64.0), J[22], y);
    y = rfma(T(4.0), J[23], y);
    s = fma(J[16].r, y.r, fma(J[16].i, y.i, s)); }
  { cplx<T> y = T(256.0) * J[17];
    y = rfma(T(4.0), J[22], y);
    s = fma(J[17].r, y.r, fma(J[17].i, y.i, s)); }
  return s;
}
template <typename T> __device__ __forceinline__ T colour_form_orbit(const cplx<T> (&J)[24]) { return colour_form_orbit_4<T>(J); }
template <> struct ColourPerm<4> {
  static __device__ __forceinline__ int at(int a) { return kColourPerm4[a]; }
};
}  // namespace mf
