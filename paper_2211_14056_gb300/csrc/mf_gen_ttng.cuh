// GENERATED by paper_2211_14056_gb300/gen_tables.py -- do not edit.
// Heavy-quark pair + n gluons: colour matrices, sub-current tables and the
// straight-line quark-line code of one helicity lane (see the generator's
// docstring for the recursion it encodes).
#pragma once
#include "mf_device.cuh"
namespace mf {
template <int NG> struct TTNG;
template <int NG, int K> __device__ __forceinline__ const uint8_t* o3_table();
template <int NG, int K> __device__ __forceinline__ const uint8_t* o4_table();
template <int NG> __device__ __forceinline__ const uint8_t* blk_mask();
template <int NG> __device__ __forceinline__ const uint16_t* blk_off();
template <typename T> __device__ __forceinline__ V4<T> neg(const V4<T>& a) {
  V4<T> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.c[k] = -a.c[k];
  return o;
}
// colour matrix, 2 gluons: C = M / 3; orderings lexicographic
static constexpr int kColourDen2 = 3;
static const int kColourNum2[4] = {16, -2, -2, 16};
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
static __constant__ uint8_t kO3_2_2[2] = {0, 1};
template <> __device__ __forceinline__ const uint8_t* o3_table<2, 2>() { return kO3_2_2; }
// One lane: fixed gluon helicities (word H) and tbar helicity (spinor vb).
// Returns sum over both top helicities of J^dagger (D C) J for the
// 2 colour orderings (integer colour matrix, D = 3).
template <typename T>
__device__ __forceinline__ T lane_colour_sum_2(const R4<T>* __restrict__ q, const R4<T>& qtb, T m, T mw,
    const V4<T>* __restrict__ Gs, unsigned H, const S4<T>& vb, const S4<T>& ub0, const S4<T>& ub1,
    cplx<T> (&J)[2][2]) {
  { S4<T> R0;
    { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), vb);
      R0 = quark_prop(R4<T>(-(qtb + q[0])), m, mw, X); }
    { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R0);
      apply_acc(make_slash(neg(Gs[4 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), vb, W);
      J[1][0] = rowdot(ub0, W); J[1][1] = rowdot(ub1, W); }
  }
  { S4<T> R1;
    { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), vb);
      R1 = quark_prop(R4<T>(-(qtb + q[1])), m, mw, X); }
    { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R1);
      apply_acc(make_slash(Gs[4 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), vb, W);
      J[0][0] = rowdot(ub0, W); J[0][1] = rowdot(ub1, W); }
  }
  T tot = T(0);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    T s = T(0);
    { cplx<T> y = T(8.0) * J[0][h];
      y = rfma(T(-2.0), J[1][h], y);
      s = fma(J[0][h].r, y.r, fma(J[0][h].i, y.i, s)); }
    { cplx<T> y = T(8.0) * J[1][h];
      s = fma(J[1][h].r, y.r, fma(J[1][h].i, y.i, s)); }
    tot += T(2) * s;
  }
  return tot;
}
// colour matrix, 3 gluons: C = M / 9; orderings lexicographic
static constexpr int kColourDen3 = 9;
static const int kColourNum3[36] = {64, -8, -8, 1, 1, 10, -8, 64, 1, 10, -8, 1, -8, 1, 64, -8, 10, 1, 1, 10, -8, 64, 1, -8, 1, -8, 10, 1, 64, -8, 10, 1, 1, -8, -8, 64};
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
static __constant__ uint8_t kO3_3_2[6] = {0, 1, 0, 2, 1, 2};
template <> __device__ __forceinline__ const uint8_t* o3_table<3, 2>() { return kO3_3_2; }
static __constant__ uint8_t kO3_3_3[12] = {0, 5, 3, 2, 0, 133, 4, 1, 1, 4, 131, 2};
template <> __device__ __forceinline__ const uint8_t* o3_table<3, 3>() { return kO3_3_3; }
static __constant__ uint8_t kO4_3_3[9] = {0, 1, 2, 0, 2, 1, 1, 0, 2};
template <> __device__ __forceinline__ const uint8_t* o4_table<3, 3>() { return kO4_3_3; }
// One lane: fixed gluon helicities (word H) and tbar helicity (spinor vb).
// Returns sum over both top helicities of J^dagger (D C) J for the
// 6 colour orderings (integer colour matrix, D = 9).
template <typename T>
__device__ __forceinline__ T lane_colour_sum_3(const R4<T>* __restrict__ q, const R4<T>& qtb, T m, T mw,
    const V4<T>* __restrict__ Gs, unsigned H, const S4<T>& vb, const S4<T>& ub0, const S4<T>& ub1,
    cplx<T> (&J)[6][2]) {
  { S4<T> R0;
    { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), vb);
      R0 = quark_prop(R4<T>(-(qtb + q[0])), m, mw, X); }
    { S4<T> R10;
      { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R0);
        apply_acc(make_slash(neg(Gs[6 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), vb, X);
        R10 = quark_prop(R4<T>(-(qtb + q[1] + q[0])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R10);
        apply_acc(make_slash(neg(Gs[14 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R0, W);
        apply_acc(make_slash(Gs[18 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[5][0] = rowdot(ub0, W); J[5][1] = rowdot(ub1, W); }
    }
    { S4<T> R20;
      { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R0);
        apply_acc(make_slash(neg(Gs[10 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), vb, X);
        R20 = quark_prop(R4<T>(-(qtb + q[2] + q[0])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R20);
        apply_acc(make_slash(Gs[14 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R0, W);
        apply_acc(make_slash(Gs[26 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[3][0] = rowdot(ub0, W); J[3][1] = rowdot(ub1, W); }
    }
  }
  { S4<T> R1;
    { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), vb);
      R1 = quark_prop(R4<T>(-(qtb + q[1])), m, mw, X); }
    { S4<T> R01;
      { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R1);
        apply_acc(make_slash(Gs[6 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), vb, X);
        R01 = quark_prop(R4<T>(-(qtb + q[0] + q[1])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R01);
        apply_acc(make_slash(neg(Gs[10 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R1, W);
        apply_acc(make_slash(Gs[34 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[4][0] = rowdot(ub0, W); J[4][1] = rowdot(ub1, W); }
    }
    { S4<T> R21;
      { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R1);
        apply_acc(make_slash(neg(Gs[14 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), vb, X);
        R21 = quark_prop(R4<T>(-(qtb + q[2] + q[1])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R21);
        apply_acc(make_slash(Gs[10 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R1, W);
        apply_acc(make_slash(Gs[26 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[1][0] = rowdot(ub0, W); J[1][1] = rowdot(ub1, W); }
    }
  }
  { S4<T> R2;
    { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), vb);
      R2 = quark_prop(R4<T>(-(qtb + q[2])), m, mw, X); }
    { S4<T> R02;
      { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R2);
        apply_acc(make_slash(Gs[10 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), vb, X);
        R02 = quark_prop(R4<T>(-(qtb + q[0] + q[2])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R02);
        apply_acc(make_slash(neg(Gs[6 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), R2, W);
        apply_acc(make_slash(Gs[34 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[2][0] = rowdot(ub0, W); J[2][1] = rowdot(ub1, W); }
    }
    { S4<T> R12;
      { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R2);
        apply_acc(make_slash(Gs[14 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), vb, X);
        R12 = quark_prop(R4<T>(-(qtb + q[1] + q[2])), m, mw, X); }
      { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R12);
        apply_acc(make_slash(Gs[6 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), R2, W);
        apply_acc(make_slash(Gs[18 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, W);
        J[0][0] = rowdot(ub0, W); J[0][1] = rowdot(ub1, W); }
    }
  }
  T tot = T(0);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    T s = T(0);
    { cplx<T> y = T(32.0) * J[0][h];
      y = rfma(T(-8.0), J[1][h], y);
      y = rfma(T(-8.0), J[2][h], y);
      y = rfma(T(1.0), J[3][h], y);
      y = rfma(T(1.0), J[4][h], y);
      y = rfma(T(10.0), J[5][h], y);
      s = fma(J[0][h].r, y.r, fma(J[0][h].i, y.i, s)); }
    { cplx<T> y = T(32.0) * J[1][h];
      y = rfma(T(1.0), J[2][h], y);
      y = rfma(T(10.0), J[3][h], y);
      y = rfma(T(-8.0), J[4][h], y);
      y = rfma(T(1.0), J[5][h], y);
      s = fma(J[1][h].r, y.r, fma(J[1][h].i, y.i, s)); }
    { cplx<T> y = T(32.0) * J[2][h];
      y = rfma(T(-8.0), J[3][h], y);
      y = rfma(T(10.0), J[4][h], y);
      y = rfma(T(1.0), J[5][h], y);
      s = fma(J[2][h].r, y.r, fma(J[2][h].i, y.i, s)); }
    { cplx<T> y = T(32.0) * J[3][h];
      y = rfma(T(1.0), J[4][h], y);
      y = rfma(T(-8.0), J[5][h], y);
      s = fma(J[3][h].r, y.r, fma(J[3][h].i, y.i, s)); }
    { cplx<T> y = T(32.0) * J[4][h];
      y = rfma(T(-8.0), J[5][h], y);
      s = fma(J[4][h].r, y.r, fma(J[4][h].i, y.i, s)); }
    { cplx<T> y = T(32.0) * J[5][h];
      s = fma(J[5][h].r, y.r, fma(J[5][h].i, y.i, s)); }
    tot += T(2) * s;
  }
  return tot;
}
// colour matrix, 4 gluons: C = M / 54; orderings lexicographic
static constexpr int kColourDen4 = 54;
static const int kColourNum4[576] = {512, -64, -64, 8, 8, 80, -64, 8, 8, -1, -1, -10, 8, -1, 80, -10, 71, 62, -1, -10, -10, 62, 62, -28, -64, 512, 8, 80, -64, 8, 8, -64, -1, -10, 8, -1, -1, -10, -10, 62, 62, -28, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, 80, -10, 71, 62, -64, 8, 8, -1, -1, -10, -10, -1, 62, -28, -10, 62, 8, 80, -64, 512, 8, -64, -1, -10, -10, 62, 62, -28, 8, -64, -1, -10, 8, -1, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, -1, 8, 71, 62, 80, -10, -10, -1, 62, -28, -10, 62, -64, 8, 8, -1, -1, -10, 80, 8, 8, -64, -64, 512, -10, -1, 62, -28, -10, 62, -1, 8, 71, 62, 80, -10, 8, -64, -1, -10, 8, -1, -64, 8, 8, -1, -1, -10, 512, -64, -64, 8, 8, 80, 80, -10, 8, -1, 62, 71, -10, 62, -1, -10, -28, 62, 8, -64, -1, -10, 8, -1, -64, 512, 8, 80, -64, 8, -10, 62, -1, -10, -28, 62, 80, -10, 8, -1, 62, 71, 8, -1, 80, -10, 71, 62, -64, 8, 512, -64, 80, 8, 8, -1, -64, 8, -10, -1, 62, -28, -10, -1, 62, -10, -1, -10, -10, 62, 62, -28, 8, 80, -64, 512, 8, -64, -1, -10, 8, -64, -1, 8, 71, 62, -1, 8, -10, 80, -1, 8, 71, 62, 80, -10, 8, -64, 80, 8, 512, -64, 62, -28, -10, -1, 62, -10, 8, -1, -64, 8, -10, -1, -10, -1, 62, -28, -10, 62, 80, 8, 8, -64, -64, 512, 71, 62, -1, 8, -10, 80, -1, -10, 8, -64, -1, 8, 8, -1, -64, 8, -10, -1, 80, -10, 8, -1, 62, 71, 512, -64, -64, 8, 8, 80, 62, -10, -28, 62, -1, -10, -1, -10, 8, -64, -1, 8, -10, 62, -1, -10, -28, 62, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, 80, -10, 8, -1, 62, 71, 8, -1, -64, 8, -10, -1, -64, 8, 512, -64, 80, 8, -28, 62, 62, -10, -10, -1, -10, 62, -1, -10, -28, 62, -1, -10, 8, -64, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, 71, 62, -1, 8, -10, 80, 62, -28, -10, -1, 62, -10, 8, -64, 80, 8, 512, -64, -1, 8, -10, -1, -64, 8, 62, -28, -10, -1, 62, -10, 71, 62, -1, 8, -10, 80, 80, 8, 8, -64, -64, 512, -10, -1, -1, 8, 8, -64, -1, 8, -10, -1, -64, 8, -10, 80, 62, 71, 8, -1, 62, -10, -28, 62, -1, -10, 512, -64, -64, 8, 8, 80, -10, -1, -1, 8, 8, -64, 62, -10, -28, 62, -1, -10, -10, 80, 62, 71, 8, -1, -64, 512, 8, 80, -64, 8, -10, 80, 62, 71, 8, -1, -1, 8, -10, -1, -64, 8, -28, 62, 62, -10, -10, -1, -64, 8, 512, -64, 80, 8, 62, -10, -28, 62, -1, -10, -10, -1, -1, 8, 8, -64, 62, 71, -10, 80, -1, 8, 8, 80, -64, 512, 8, -64, 62, 71, -10, 80, -1, 8, -28, 62, 62, -10, -10, -1, -1, 8, -10, -1, -64, 8, 8, -64, 80, 8, 512, -64, -28, 62, 62, -10, -10, -1, 62, 71, -10, 80, -1, 8, -10, -1, -1, 8, 8, -64, 80, 8, 8, -64, -64, 512};
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
static __constant__ uint8_t kO3_4_2[12] = {0, 1, 0, 2, 0, 3, 1, 2, 1, 3, 2, 3};
template <> __device__ __forceinline__ const uint8_t* o3_table<4, 2>() { return kO3_4_2; }
static __constant__ uint8_t kO3_4_3[48] = {0, 7, 4, 2, 0, 8, 4, 3, 0, 135, 5, 1, 0, 9, 5, 3, 0, 136, 6, 1, 0, 137, 6, 2, 1, 5, 132, 2, 1, 6, 132, 3, 1, 9, 7, 3, 1, 137, 8, 2, 2, 6, 133, 3, 2, 8, 135, 3};
template <> __device__ __forceinline__ const uint8_t* o3_table<4, 3>() { return kO3_4_3; }
static __constant__ uint8_t kO4_4_3[36] = {0, 1, 2, 0, 1, 3, 0, 2, 1, 0, 2, 3, 0, 3, 1, 0, 3, 2, 1, 0, 2, 1, 0, 3, 1, 2, 3, 1, 3, 2, 2, 0, 3, 2, 1, 3};
template <> __device__ __forceinline__ const uint8_t* o4_table<4, 3>() { return kO4_4_3; }
static __constant__ uint8_t kO3_4_4[72] = {0, 18, 4, 9, 10, 3, 0, 19, 4, 137, 11, 2, 0, 21, 5, 8, 12, 3, 0, 19, 5, 136, 13, 1, 0, 21, 6, 7, 14, 2, 0, 18, 6, 135, 15, 1, 1, 13, 132, 9, 16, 3, 1, 15, 132, 137, 17, 2, 1, 20, 7, 6, 12, 3, 1, 20, 8, 5, 14, 2, 2, 11, 133, 8, 16, 3, 2, 17, 135, 6, 10, 3};
template <> __device__ __forceinline__ const uint8_t* o3_table<4, 4>() { return kO3_4_4; }
static __constant__ uint8_t kO4_4_4[108] = {0, 1, 9, 0, 7, 3, 4, 2, 3, 0, 1, 137, 0, 8, 2, 4, 3, 2, 0, 2, 8, 0, 135, 3, 5, 1, 3, 0, 2, 136, 0, 9, 1, 5, 3, 1, 0, 3, 7, 0, 136, 2, 6, 1, 2, 0, 3, 135, 0, 137, 1, 6, 2, 1, 1, 0, 9, 1, 5, 3, 132, 2, 3, 1, 0, 137, 1, 6, 2, 132, 3, 2, 1, 2, 6, 1, 133, 3, 7, 0, 3, 1, 3, 5, 1, 134, 2, 8, 0, 2, 2, 0, 8, 2, 4, 3, 133, 1, 3, 2, 1, 6, 2, 132, 3, 135, 0, 3};
template <> __device__ __forceinline__ const uint8_t* o4_table<4, 4>() { return kO4_4_4; }
// One lane: fixed gluon helicities (word H) and tbar helicity (spinor vb).
// Returns sum over both top helicities of J^dagger (D C) J for the
// 24 colour orderings (integer colour matrix, D = 54).
template <typename T>
__device__ __forceinline__ T lane_colour_sum_4(const R4<T>* __restrict__ q, const R4<T>& qtb, T m, T mw,
    const V4<T>* __restrict__ Gs, unsigned H, const S4<T>& vb, const S4<T>& ub0, const S4<T>& ub1,
    cplx<T> (&J)[24][2]) {
  { S4<T> R0;
    { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), vb);
      R0 = quark_prop(R4<T>(-(qtb + q[0])), m, mw, X); }
    { S4<T> R10;
      { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R0);
        apply_acc(make_slash(neg(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), vb, X);
        R10 = quark_prop(R4<T>(-(qtb + q[1] + q[0])), m, mw, X); }
      { S4<T> R210;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R10);
          apply_acc(make_slash(neg(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R0, X);
          apply_acc(make_slash(Gs[32 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R210 = quark_prop(R4<T>(-(qtb + q[2] + q[1] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R210);
          apply_acc(make_slash(neg(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R10, W);
          apply_acc(make_slash(Gs[96 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[128 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[23][0] = rowdot(ub0, W); J[23][1] = rowdot(ub1, W); }
      }
      { S4<T> R310;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R10);
          apply_acc(make_slash(neg(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R0, X);
          apply_acc(make_slash(Gs[40 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R310 = quark_prop(R4<T>(-(qtb + q[3] + q[1] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R310);
          apply_acc(make_slash(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R10, W);
          apply_acc(make_slash(Gs[104 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[144 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[17][0] = rowdot(ub0, W); J[17][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R20;
      { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R0);
        apply_acc(make_slash(neg(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), vb, X);
        R20 = quark_prop(R4<T>(-(qtb + q[2] + q[0])), m, mw, X); }
      { S4<T> R120;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R20);
          apply_acc(make_slash(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R0, X);
          apply_acc(make_slash(Gs[48 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R120 = quark_prop(R4<T>(-(qtb + q[1] + q[2] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R120);
          apply_acc(make_slash(neg(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R20, W);
          apply_acc(make_slash(Gs[120 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[160 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[21][0] = rowdot(ub0, W); J[21][1] = rowdot(ub1, W); }
      }
      { S4<T> R320;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R20);
          apply_acc(make_slash(neg(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R0, X);
          apply_acc(make_slash(Gs[56 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R320 = quark_prop(R4<T>(-(qtb + q[3] + q[2] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R320);
          apply_acc(make_slash(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R20, W);
          apply_acc(make_slash(Gs[104 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[176 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[11][0] = rowdot(ub0, W); J[11][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R30;
      { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R0);
        apply_acc(make_slash(neg(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), vb, X);
        R30 = quark_prop(R4<T>(-(qtb + q[3] + q[0])), m, mw, X); }
      { S4<T> R130;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R30);
          apply_acc(make_slash(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R0, X);
          apply_acc(make_slash(Gs[64 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R130 = quark_prop(R4<T>(-(qtb + q[1] + q[3] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R130);
          apply_acc(make_slash(neg(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R30, W);
          apply_acc(make_slash(Gs[120 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[192 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[15][0] = rowdot(ub0, W); J[15][1] = rowdot(ub1, W); }
      }
      { S4<T> R230;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R30);
          apply_acc(make_slash(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R0, X);
          apply_acc(make_slash(Gs[72 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R230 = quark_prop(R4<T>(-(qtb + q[2] + q[3] + q[0])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R230);
          apply_acc(make_slash(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R30, W);
          apply_acc(make_slash(Gs[96 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R0, W);
          apply_acc(make_slash(neg(Gs[208 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[9][0] = rowdot(ub0, W); J[9][1] = rowdot(ub1, W); }
      }
    }
  }
  { S4<T> R1;
    { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), vb);
      R1 = quark_prop(R4<T>(-(qtb + q[1])), m, mw, X); }
    { S4<T> R01;
      { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R1);
        apply_acc(make_slash(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), vb, X);
        R01 = quark_prop(R4<T>(-(qtb + q[0] + q[1])), m, mw, X); }
      { S4<T> R201;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R01);
          apply_acc(make_slash(neg(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R1, X);
          apply_acc(make_slash(Gs[80 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R201 = quark_prop(R4<T>(-(qtb + q[2] + q[0] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R201);
          apply_acc(make_slash(neg(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R01, W);
          apply_acc(make_slash(Gs[56 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(neg(Gs[224 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[22][0] = rowdot(ub0, W); J[22][1] = rowdot(ub1, W); }
      }
      { S4<T> R301;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R01);
          apply_acc(make_slash(neg(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R1, X);
          apply_acc(make_slash(Gs[88 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R301 = quark_prop(R4<T>(-(qtb + q[3] + q[0] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R301);
          apply_acc(make_slash(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R01, W);
          apply_acc(make_slash(Gs[72 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(neg(Gs[240 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[16][0] = rowdot(ub0, W); J[16][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R21;
      { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R1);
        apply_acc(make_slash(neg(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), vb, X);
        R21 = quark_prop(R4<T>(-(qtb + q[2] + q[1])), m, mw, X); }
      { S4<T> R021;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R21);
          apply_acc(make_slash(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R1, X);
          apply_acc(make_slash(Gs[48 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R021 = quark_prop(R4<T>(-(qtb + q[0] + q[2] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R021);
          apply_acc(make_slash(neg(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R21, W);
          apply_acc(make_slash(Gs[112 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(neg(Gs[256 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[19][0] = rowdot(ub0, W); J[19][1] = rowdot(ub1, W); }
      }
      { S4<T> R321;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R21);
          apply_acc(make_slash(neg(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R1, X);
          apply_acc(make_slash(Gs[96 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R321 = quark_prop(R4<T>(-(qtb + q[3] + q[2] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R321);
          apply_acc(make_slash(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R21, W);
          apply_acc(make_slash(Gs[72 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(Gs[208 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[5][0] = rowdot(ub0, W); J[5][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R31;
      { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R1);
        apply_acc(make_slash(neg(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), vb, X);
        R31 = quark_prop(R4<T>(-(qtb + q[3] + q[1])), m, mw, X); }
      { S4<T> R031;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R31);
          apply_acc(make_slash(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R1, X);
          apply_acc(make_slash(Gs[64 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R031 = quark_prop(R4<T>(-(qtb + q[0] + q[3] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R031);
          apply_acc(make_slash(neg(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R31, W);
          apply_acc(make_slash(Gs[112 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(neg(Gs[272 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[13][0] = rowdot(ub0, W); J[13][1] = rowdot(ub1, W); }
      }
      { S4<T> R231;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R31);
          apply_acc(make_slash(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R1, X);
          apply_acc(make_slash(Gs[104 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R231 = quark_prop(R4<T>(-(qtb + q[2] + q[3] + q[1])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R231);
          apply_acc(make_slash(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R31, W);
          apply_acc(make_slash(Gs[56 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R1, W);
          apply_acc(make_slash(Gs[176 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[3][0] = rowdot(ub0, W); J[3][1] = rowdot(ub1, W); }
      }
    }
  }
  { S4<T> R2;
    { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), vb);
      R2 = quark_prop(R4<T>(-(qtb + q[2])), m, mw, X); }
    { S4<T> R02;
      { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R2);
        apply_acc(make_slash(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), vb, X);
        R02 = quark_prop(R4<T>(-(qtb + q[0] + q[2])), m, mw, X); }
      { S4<T> R102;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R02);
          apply_acc(make_slash(neg(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), R2, X);
          apply_acc(make_slash(Gs[80 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R102 = quark_prop(R4<T>(-(qtb + q[1] + q[0] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R102);
          apply_acc(make_slash(neg(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R02, W);
          apply_acc(make_slash(Gs[40 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(neg(Gs[288 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[20][0] = rowdot(ub0, W); J[20][1] = rowdot(ub1, W); }
      }
      { S4<T> R302;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R02);
          apply_acc(make_slash(neg(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R2, X);
          apply_acc(make_slash(Gs[112 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R302 = quark_prop(R4<T>(-(qtb + q[3] + q[0] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R302);
          apply_acc(make_slash(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R02, W);
          apply_acc(make_slash(Gs[64 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(Gs[272 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[10][0] = rowdot(ub0, W); J[10][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R12;
      { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R2);
        apply_acc(make_slash(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), vb, X);
        R12 = quark_prop(R4<T>(-(qtb + q[1] + q[2])), m, mw, X); }
      { S4<T> R012;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R12);
          apply_acc(make_slash(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), R2, X);
          apply_acc(make_slash(Gs[32 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), vb, X);
          R012 = quark_prop(R4<T>(-(qtb + q[0] + q[1] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R012);
          apply_acc(make_slash(neg(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R12, W);
          apply_acc(make_slash(Gs[88 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(neg(Gs[304 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))])), vb, W);
          J[18][0] = rowdot(ub0, W); J[18][1] = rowdot(ub1, W); }
      }
      { S4<T> R312;
        { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R12);
          apply_acc(make_slash(neg(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), R2, X);
          apply_acc(make_slash(Gs[120 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R312 = quark_prop(R4<T>(-(qtb + q[3] + q[1] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R312);
          apply_acc(make_slash(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R12, W);
          apply_acc(make_slash(Gs[64 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(Gs[192 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[4][0] = rowdot(ub0, W); J[4][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R32;
      { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), R2);
        apply_acc(make_slash(neg(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))])), vb, X);
        R32 = quark_prop(R4<T>(-(qtb + q[3] + q[2])), m, mw, X); }
      { S4<T> R032;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R32);
          apply_acc(make_slash(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R2, X);
          apply_acc(make_slash(Gs[72 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R032 = quark_prop(R4<T>(-(qtb + q[0] + q[3] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R032);
          apply_acc(make_slash(neg(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), R32, W);
          apply_acc(make_slash(Gs[88 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(Gs[240 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[7][0] = rowdot(ub0, W); J[7][1] = rowdot(ub1, W); }
      }
      { S4<T> R132;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R32);
          apply_acc(make_slash(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), R2, X);
          apply_acc(make_slash(Gs[104 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R132 = quark_prop(R4<T>(-(qtb + q[1] + q[3] + q[2])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R132);
          apply_acc(make_slash(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), R32, W);
          apply_acc(make_slash(Gs[40 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), R2, W);
          apply_acc(make_slash(Gs[144 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[1][0] = rowdot(ub0, W); J[1][1] = rowdot(ub1, W); }
      }
    }
  }
  { S4<T> R3;
    { S4<T> X = apply(make_slash(Gs[6 + ((((H >> 3) & 1u) << 0))]), vb);
      R3 = quark_prop(R4<T>(-(qtb + q[3])), m, mw, X); }
    { S4<T> R03;
      { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R3);
        apply_acc(make_slash(Gs[16 + ((((H >> 0) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), vb, X);
        R03 = quark_prop(R4<T>(-(qtb + q[0] + q[3])), m, mw, X); }
      { S4<T> R103;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R03);
          apply_acc(make_slash(neg(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), R3, X);
          apply_acc(make_slash(Gs[88 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R103 = quark_prop(R4<T>(-(qtb + q[1] + q[0] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R103);
          apply_acc(make_slash(neg(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R03, W);
          apply_acc(make_slash(Gs[32 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[304 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[14][0] = rowdot(ub0, W); J[14][1] = rowdot(ub1, W); }
      }
      { S4<T> R203;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R03);
          apply_acc(make_slash(neg(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R3, X);
          apply_acc(make_slash(Gs[112 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R203 = quark_prop(R4<T>(-(qtb + q[2] + q[0] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R203);
          apply_acc(make_slash(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R03, W);
          apply_acc(make_slash(Gs[48 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[256 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[8][0] = rowdot(ub0, W); J[8][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R13;
      { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R3);
        apply_acc(make_slash(Gs[24 + ((((H >> 1) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), vb, X);
        R13 = quark_prop(R4<T>(-(qtb + q[1] + q[3])), m, mw, X); }
      { S4<T> R013;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R13);
          apply_acc(make_slash(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), R3, X);
          apply_acc(make_slash(Gs[40 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R013 = quark_prop(R4<T>(-(qtb + q[0] + q[1] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R013);
          apply_acc(make_slash(neg(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R13, W);
          apply_acc(make_slash(Gs[80 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[288 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[12][0] = rowdot(ub0, W); J[12][1] = rowdot(ub1, W); }
      }
      { S4<T> R213;
        { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R13);
          apply_acc(make_slash(neg(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))])), R3, X);
          apply_acc(make_slash(Gs[120 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R213 = quark_prop(R4<T>(-(qtb + q[2] + q[1] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R213);
          apply_acc(make_slash(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R13, W);
          apply_acc(make_slash(Gs[48 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[160 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[2][0] = rowdot(ub0, W); J[2][1] = rowdot(ub1, W); }
      }
    }
    { S4<T> R23;
      { S4<T> X = apply(make_slash(Gs[4 + ((((H >> 2) & 1u) << 0))]), R3);
        apply_acc(make_slash(Gs[28 + ((((H >> 2) & 1u) << 0) | (((H >> 3) & 1u) << 1))]), vb, X);
        R23 = quark_prop(R4<T>(-(qtb + q[2] + q[3])), m, mw, X); }
      { S4<T> R023;
        { S4<T> X = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R23);
          apply_acc(make_slash(Gs[12 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R3, X);
          apply_acc(make_slash(Gs[56 + ((((H >> 0) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R023 = quark_prop(R4<T>(-(qtb + q[0] + q[2] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R023);
          apply_acc(make_slash(neg(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))])), R23, W);
          apply_acc(make_slash(Gs[80 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[224 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[6][0] = rowdot(ub0, W); J[6][1] = rowdot(ub1, W); }
      }
      { S4<T> R123;
        { S4<T> X = apply(make_slash(Gs[2 + ((((H >> 1) & 1u) << 0))]), R23);
          apply_acc(make_slash(Gs[20 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1))]), R3, X);
          apply_acc(make_slash(Gs[96 + ((((H >> 1) & 1u) << 0) | (((H >> 2) & 1u) << 1) | (((H >> 3) & 1u) << 2))]), vb, X);
          R123 = quark_prop(R4<T>(-(qtb + q[1] + q[2] + q[3])), m, mw, X); }
        { S4<T> W = apply(make_slash(Gs[0 + ((((H >> 0) & 1u) << 0))]), R123);
          apply_acc(make_slash(Gs[8 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1))]), R23, W);
          apply_acc(make_slash(Gs[32 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2))]), R3, W);
          apply_acc(make_slash(Gs[128 + ((((H >> 0) & 1u) << 0) | (((H >> 1) & 1u) << 1) | (((H >> 2) & 1u) << 2) | (((H >> 3) & 1u) << 3))]), vb, W);
          J[0][0] = rowdot(ub0, W); J[0][1] = rowdot(ub1, W); }
      }
    }
  }
  T tot = T(0);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    T s = T(0);
    { cplx<T> y = T(256.0) * J[0][h];
      y = rfma(T(-64.0), J[1][h], y);
      y = rfma(T(-64.0), J[2][h], y);
      y = rfma(T(8.0), J[3][h], y);
      y = rfma(T(8.0), J[4][h], y);
      y = rfma(T(80.0), J[5][h], y);
      y = rfma(T(-64.0), J[6][h], y);
      y = rfma(T(8.0), J[7][h], y);
      y = rfma(T(8.0), J[8][h], y);
      y = rfma(T(-1.0), J[9][h], y);
      y = rfma(T(-1.0), J[10][h], y);
      y = rfma(T(-10.0), J[11][h], y);
      y = rfma(T(8.0), J[12][h], y);
      y = rfma(T(-1.0), J[13][h], y);
      y = rfma(T(80.0), J[14][h], y);
      y = rfma(T(-10.0), J[15][h], y);
      y = rfma(T(71.0), J[16][h], y);
      y = rfma(T(62.0), J[17][h], y);
      y = rfma(T(-1.0), J[18][h], y);
      y = rfma(T(-10.0), J[19][h], y);
      y = rfma(T(-10.0), J[20][h], y);
      y = rfma(T(62.0), J[21][h], y);
      y = rfma(T(62.0), J[22][h], y);
      y = rfma(T(-28.0), J[23][h], y);
      s = fma(J[0][h].r, y.r, fma(J[0][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[1][h];
      y = rfma(T(8.0), J[2][h], y);
      y = rfma(T(80.0), J[3][h], y);
      y = rfma(T(-64.0), J[4][h], y);
      y = rfma(T(8.0), J[5][h], y);
      y = rfma(T(8.0), J[6][h], y);
      y = rfma(T(-64.0), J[7][h], y);
      y = rfma(T(-1.0), J[8][h], y);
      y = rfma(T(-10.0), J[9][h], y);
      y = rfma(T(8.0), J[10][h], y);
      y = rfma(T(-1.0), J[11][h], y);
      y = rfma(T(-1.0), J[12][h], y);
      y = rfma(T(-10.0), J[13][h], y);
      y = rfma(T(-10.0), J[14][h], y);
      y = rfma(T(62.0), J[15][h], y);
      y = rfma(T(62.0), J[16][h], y);
      y = rfma(T(-28.0), J[17][h], y);
      y = rfma(T(8.0), J[18][h], y);
      y = rfma(T(-1.0), J[19][h], y);
      y = rfma(T(80.0), J[20][h], y);
      y = rfma(T(-10.0), J[21][h], y);
      y = rfma(T(71.0), J[22][h], y);
      y = rfma(T(62.0), J[23][h], y);
      s = fma(J[1][h].r, y.r, fma(J[1][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[2][h];
      y = rfma(T(-64.0), J[3][h], y);
      y = rfma(T(80.0), J[4][h], y);
      y = rfma(T(8.0), J[5][h], y);
      y = rfma(T(8.0), J[6][h], y);
      y = rfma(T(-1.0), J[7][h], y);
      y = rfma(T(80.0), J[8][h], y);
      y = rfma(T(-10.0), J[9][h], y);
      y = rfma(T(71.0), J[10][h], y);
      y = rfma(T(62.0), J[11][h], y);
      y = rfma(T(-64.0), J[12][h], y);
      y = rfma(T(8.0), J[13][h], y);
      y = rfma(T(8.0), J[14][h], y);
      y = rfma(T(-1.0), J[15][h], y);
      y = rfma(T(-1.0), J[16][h], y);
      y = rfma(T(-10.0), J[17][h], y);
      y = rfma(T(-10.0), J[18][h], y);
      y = rfma(T(-1.0), J[19][h], y);
      y = rfma(T(62.0), J[20][h], y);
      y = rfma(T(-28.0), J[21][h], y);
      y = rfma(T(-10.0), J[22][h], y);
      y = rfma(T(62.0), J[23][h], y);
      s = fma(J[2][h].r, y.r, fma(J[2][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[3][h];
      y = rfma(T(8.0), J[4][h], y);
      y = rfma(T(-64.0), J[5][h], y);
      y = rfma(T(-1.0), J[6][h], y);
      y = rfma(T(-10.0), J[7][h], y);
      y = rfma(T(-10.0), J[8][h], y);
      y = rfma(T(62.0), J[9][h], y);
      y = rfma(T(62.0), J[10][h], y);
      y = rfma(T(-28.0), J[11][h], y);
      y = rfma(T(8.0), J[12][h], y);
      y = rfma(T(-64.0), J[13][h], y);
      y = rfma(T(-1.0), J[14][h], y);
      y = rfma(T(-10.0), J[15][h], y);
      y = rfma(T(8.0), J[16][h], y);
      y = rfma(T(-1.0), J[17][h], y);
      y = rfma(T(-1.0), J[18][h], y);
      y = rfma(T(8.0), J[19][h], y);
      y = rfma(T(71.0), J[20][h], y);
      y = rfma(T(62.0), J[21][h], y);
      y = rfma(T(80.0), J[22][h], y);
      y = rfma(T(-10.0), J[23][h], y);
      s = fma(J[3][h].r, y.r, fma(J[3][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[4][h];
      y = rfma(T(-64.0), J[5][h], y);
      y = rfma(T(-1.0), J[6][h], y);
      y = rfma(T(8.0), J[7][h], y);
      y = rfma(T(71.0), J[8][h], y);
      y = rfma(T(62.0), J[9][h], y);
      y = rfma(T(80.0), J[10][h], y);
      y = rfma(T(-10.0), J[11][h], y);
      y = rfma(T(-10.0), J[12][h], y);
      y = rfma(T(-1.0), J[13][h], y);
      y = rfma(T(62.0), J[14][h], y);
      y = rfma(T(-28.0), J[15][h], y);
      y = rfma(T(-10.0), J[16][h], y);
      y = rfma(T(62.0), J[17][h], y);
      y = rfma(T(-64.0), J[18][h], y);
      y = rfma(T(8.0), J[19][h], y);
      y = rfma(T(8.0), J[20][h], y);
      y = rfma(T(-1.0), J[21][h], y);
      y = rfma(T(-1.0), J[22][h], y);
      y = rfma(T(-10.0), J[23][h], y);
      s = fma(J[4][h].r, y.r, fma(J[4][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[5][h];
      y = rfma(T(-10.0), J[6][h], y);
      y = rfma(T(-1.0), J[7][h], y);
      y = rfma(T(62.0), J[8][h], y);
      y = rfma(T(-28.0), J[9][h], y);
      y = rfma(T(-10.0), J[10][h], y);
      y = rfma(T(62.0), J[11][h], y);
      y = rfma(T(-1.0), J[12][h], y);
      y = rfma(T(8.0), J[13][h], y);
      y = rfma(T(71.0), J[14][h], y);
      y = rfma(T(62.0), J[15][h], y);
      y = rfma(T(80.0), J[16][h], y);
      y = rfma(T(-10.0), J[17][h], y);
      y = rfma(T(8.0), J[18][h], y);
      y = rfma(T(-64.0), J[19][h], y);
      y = rfma(T(-1.0), J[20][h], y);
      y = rfma(T(-10.0), J[21][h], y);
      y = rfma(T(8.0), J[22][h], y);
      y = rfma(T(-1.0), J[23][h], y);
      s = fma(J[5][h].r, y.r, fma(J[5][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[6][h];
      y = rfma(T(-64.0), J[7][h], y);
      y = rfma(T(-64.0), J[8][h], y);
      y = rfma(T(8.0), J[9][h], y);
      y = rfma(T(8.0), J[10][h], y);
      y = rfma(T(80.0), J[11][h], y);
      y = rfma(T(80.0), J[12][h], y);
      y = rfma(T(-10.0), J[13][h], y);
      y = rfma(T(8.0), J[14][h], y);
      y = rfma(T(-1.0), J[15][h], y);
      y = rfma(T(62.0), J[16][h], y);
      y = rfma(T(71.0), J[17][h], y);
      y = rfma(T(-10.0), J[18][h], y);
      y = rfma(T(62.0), J[19][h], y);
      y = rfma(T(-1.0), J[20][h], y);
      y = rfma(T(-10.0), J[21][h], y);
      y = rfma(T(-28.0), J[22][h], y);
      y = rfma(T(62.0), J[23][h], y);
      s = fma(J[6][h].r, y.r, fma(J[6][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[7][h];
      y = rfma(T(8.0), J[8][h], y);
      y = rfma(T(80.0), J[9][h], y);
      y = rfma(T(-64.0), J[10][h], y);
      y = rfma(T(8.0), J[11][h], y);
      y = rfma(T(-10.0), J[12][h], y);
      y = rfma(T(62.0), J[13][h], y);
      y = rfma(T(-1.0), J[14][h], y);
      y = rfma(T(-10.0), J[15][h], y);
      y = rfma(T(-28.0), J[16][h], y);
      y = rfma(T(62.0), J[17][h], y);
      y = rfma(T(80.0), J[18][h], y);
      y = rfma(T(-10.0), J[19][h], y);
      y = rfma(T(8.0), J[20][h], y);
      y = rfma(T(-1.0), J[21][h], y);
      y = rfma(T(62.0), J[22][h], y);
      y = rfma(T(71.0), J[23][h], y);
      s = fma(J[7][h].r, y.r, fma(J[7][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[8][h];
      y = rfma(T(-64.0), J[9][h], y);
      y = rfma(T(80.0), J[10][h], y);
      y = rfma(T(8.0), J[11][h], y);
      y = rfma(T(8.0), J[12][h], y);
      y = rfma(T(-1.0), J[13][h], y);
      y = rfma(T(-64.0), J[14][h], y);
      y = rfma(T(8.0), J[15][h], y);
      y = rfma(T(-10.0), J[16][h], y);
      y = rfma(T(-1.0), J[17][h], y);
      y = rfma(T(62.0), J[18][h], y);
      y = rfma(T(-28.0), J[19][h], y);
      y = rfma(T(-10.0), J[20][h], y);
      y = rfma(T(-1.0), J[21][h], y);
      y = rfma(T(62.0), J[22][h], y);
      y = rfma(T(-10.0), J[23][h], y);
      s = fma(J[8][h].r, y.r, fma(J[8][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[9][h];
      y = rfma(T(8.0), J[10][h], y);
      y = rfma(T(-64.0), J[11][h], y);
      y = rfma(T(-1.0), J[12][h], y);
      y = rfma(T(-10.0), J[13][h], y);
      y = rfma(T(8.0), J[14][h], y);
      y = rfma(T(-64.0), J[15][h], y);
      y = rfma(T(-1.0), J[16][h], y);
      y = rfma(T(8.0), J[17][h], y);
      y = rfma(T(71.0), J[18][h], y);
      y = rfma(T(62.0), J[19][h], y);
      y = rfma(T(-1.0), J[20][h], y);
      y = rfma(T(8.0), J[21][h], y);
      y = rfma(T(-10.0), J[22][h], y);
      y = rfma(T(80.0), J[23][h], y);
      s = fma(J[9][h].r, y.r, fma(J[9][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[10][h];
      y = rfma(T(-64.0), J[11][h], y);
      y = rfma(T(62.0), J[12][h], y);
      y = rfma(T(-28.0), J[13][h], y);
      y = rfma(T(-10.0), J[14][h], y);
      y = rfma(T(-1.0), J[15][h], y);
      y = rfma(T(62.0), J[16][h], y);
      y = rfma(T(-10.0), J[17][h], y);
      y = rfma(T(8.0), J[18][h], y);
      y = rfma(T(-1.0), J[19][h], y);
      y = rfma(T(-64.0), J[20][h], y);
      y = rfma(T(8.0), J[21][h], y);
      y = rfma(T(-10.0), J[22][h], y);
      y = rfma(T(-1.0), J[23][h], y);
      s = fma(J[10][h].r, y.r, fma(J[10][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[11][h];
      y = rfma(T(71.0), J[12][h], y);
      y = rfma(T(62.0), J[13][h], y);
      y = rfma(T(-1.0), J[14][h], y);
      y = rfma(T(8.0), J[15][h], y);
      y = rfma(T(-10.0), J[16][h], y);
      y = rfma(T(80.0), J[17][h], y);
      y = rfma(T(-1.0), J[18][h], y);
      y = rfma(T(-10.0), J[19][h], y);
      y = rfma(T(8.0), J[20][h], y);
      y = rfma(T(-64.0), J[21][h], y);
      y = rfma(T(-1.0), J[22][h], y);
      y = rfma(T(8.0), J[23][h], y);
      s = fma(J[11][h].r, y.r, fma(J[11][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[12][h];
      y = rfma(T(-64.0), J[13][h], y);
      y = rfma(T(-64.0), J[14][h], y);
      y = rfma(T(8.0), J[15][h], y);
      y = rfma(T(8.0), J[16][h], y);
      y = rfma(T(80.0), J[17][h], y);
      y = rfma(T(62.0), J[18][h], y);
      y = rfma(T(-10.0), J[19][h], y);
      y = rfma(T(-28.0), J[20][h], y);
      y = rfma(T(62.0), J[21][h], y);
      y = rfma(T(-1.0), J[22][h], y);
      y = rfma(T(-10.0), J[23][h], y);
      s = fma(J[12][h].r, y.r, fma(J[12][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[13][h];
      y = rfma(T(8.0), J[14][h], y);
      y = rfma(T(80.0), J[15][h], y);
      y = rfma(T(-64.0), J[16][h], y);
      y = rfma(T(8.0), J[17][h], y);
      y = rfma(T(-10.0), J[18][h], y);
      y = rfma(T(80.0), J[19][h], y);
      y = rfma(T(62.0), J[20][h], y);
      y = rfma(T(71.0), J[21][h], y);
      y = rfma(T(8.0), J[22][h], y);
      y = rfma(T(-1.0), J[23][h], y);
      s = fma(J[13][h].r, y.r, fma(J[13][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[14][h];
      y = rfma(T(-64.0), J[15][h], y);
      y = rfma(T(80.0), J[16][h], y);
      y = rfma(T(8.0), J[17][h], y);
      y = rfma(T(-28.0), J[18][h], y);
      y = rfma(T(62.0), J[19][h], y);
      y = rfma(T(62.0), J[20][h], y);
      y = rfma(T(-10.0), J[21][h], y);
      y = rfma(T(-10.0), J[22][h], y);
      y = rfma(T(-1.0), J[23][h], y);
      s = fma(J[14][h].r, y.r, fma(J[14][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[15][h];
      y = rfma(T(8.0), J[16][h], y);
      y = rfma(T(-64.0), J[17][h], y);
      y = rfma(T(62.0), J[18][h], y);
      y = rfma(T(71.0), J[19][h], y);
      y = rfma(T(-10.0), J[20][h], y);
      y = rfma(T(80.0), J[21][h], y);
      y = rfma(T(-1.0), J[22][h], y);
      y = rfma(T(8.0), J[23][h], y);
      s = fma(J[15][h].r, y.r, fma(J[15][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[16][h];
      y = rfma(T(-64.0), J[17][h], y);
      y = rfma(T(-1.0), J[18][h], y);
      y = rfma(T(8.0), J[19][h], y);
      y = rfma(T(-10.0), J[20][h], y);
      y = rfma(T(-1.0), J[21][h], y);
      y = rfma(T(-64.0), J[22][h], y);
      y = rfma(T(8.0), J[23][h], y);
      s = fma(J[16][h].r, y.r, fma(J[16][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[17][h];
      y = rfma(T(-10.0), J[18][h], y);
      y = rfma(T(-1.0), J[19][h], y);
      y = rfma(T(-1.0), J[20][h], y);
      y = rfma(T(8.0), J[21][h], y);
      y = rfma(T(8.0), J[22][h], y);
      y = rfma(T(-64.0), J[23][h], y);
      s = fma(J[17][h].r, y.r, fma(J[17][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[18][h];
      y = rfma(T(-64.0), J[19][h], y);
      y = rfma(T(-64.0), J[20][h], y);
      y = rfma(T(8.0), J[21][h], y);
      y = rfma(T(8.0), J[22][h], y);
      y = rfma(T(80.0), J[23][h], y);
      s = fma(J[18][h].r, y.r, fma(J[18][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[19][h];
      y = rfma(T(8.0), J[20][h], y);
      y = rfma(T(80.0), J[21][h], y);
      y = rfma(T(-64.0), J[22][h], y);
      y = rfma(T(8.0), J[23][h], y);
      s = fma(J[19][h].r, y.r, fma(J[19][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[20][h];
      y = rfma(T(-64.0), J[21][h], y);
      y = rfma(T(80.0), J[22][h], y);
      y = rfma(T(8.0), J[23][h], y);
      s = fma(J[20][h].r, y.r, fma(J[20][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[21][h];
      y = rfma(T(8.0), J[22][h], y);
      y = rfma(T(-64.0), J[23][h], y);
      s = fma(J[21][h].r, y.r, fma(J[21][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[22][h];
      y = rfma(T(-64.0), J[23][h], y);
      s = fma(J[22][h].r, y.r, fma(J[22][h].i, y.i, s)); }
    { cplx<T> y = T(256.0) * J[23][h];
      s = fma(J[23][h].r, y.r, fma(J[23][h].i, y.i, s)); }
    tot += T(2) * s;
  }
  return tot;
}
}  // namespace mf
