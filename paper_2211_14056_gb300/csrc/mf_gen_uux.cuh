// GENERATED by paper_2211_14056_gb300/gen_uux.py -- do not edit.
// u u~ -> t t~ g g: tree diagrams, colour decomposition onto 12 structures,
// straight-line code of one helicity configuration (see the generator's docstring).
#pragma once
#include "mf_uux.cuh"
namespace mf {
constexpr int kUuxFlows = 12;
static constexpr int kUuxColourDen = 3;
static const int kUuxColourNum[144] = {48, -6, 0, 0, 6, 6, 16, -2, -2, 16, 16, -2, -6, 48, 0, 0, 6, 6, -2, 16, 16, -2, -2, 16, 0, 0, 48, 6, 0, 0, -2, 16, 16, 16, 16, -2, 0, 0, 6, 48, 0, 0, 16, -2, 16, 16, -2, 16, 6, 6, 0, 0, 48, -6, 16, -2, 16, -2, 16, -2, 6, 6, 0, 0, -6, 48, -2, 16, -2, 16, -2, 16, 16, -2, -2, 16, 16, -2, 48, -6, 0, 0, 6, 6, -2, 16, 16, -2, -2, 16, -6, 48, 0, 0, 6, 6, -2, 16, 16, 16, 16, -2, 0, 0, 48, 6, 0, 0, 16, -2, 16, 16, -2, 16, 0, 0, 6, 48, 0, 0, 16, -2, 16, -2, 16, -2, 6, 6, 0, 0, 48, -6, -2, 16, -2, 16, -2, 16, 6, 6, 0, 0, -6, 48};
// 38 diagrams; colour basis: tu A=() B=(5, 6); tu A=() B=(6, 5); tu A=(5,) B=(6,); tu A=(6,) B=(5,); tu A=(5, 6) B=(); tu A=(6, 5) B=(); tt A=() B=(5, 6); tt A=() B=(6, 5); tt A=(5,) B=(6,); tt A=(6,) B=(5,); tt A=(5, 6) B=(); tt A=(6, 5) B=()
template <typename T>
__device__ __forceinline__ void uux_amplitudes(const R4<T> (&p)[6], T mt, T mw, const S4<T>& U1, const S4<T>& V2, const S4<T>& VTB, const S4<T> (&UB3)[2], const V4<T>& E5, const V4<T>& E6, cplx<T> (&J)[2][12]) {
  R4<T> K0;
#pragma unroll
  for (int c = 0; c < 4; ++c) K0.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c];
  R4<T> K1;
#pragma unroll
  for (int c = 0; c < 4; ++c) K1.v[c] = T(-1) * p[3].v[c] + T(-1) * p[5].v[c];
  R4<T> K2;
#pragma unroll
  for (int c = 0; c < 4; ++c) K2.v[c] = T(-1) * p[3].v[c] + T(-1) * p[4].v[c] + T(-1) * p[5].v[c];
  R4<T> K3;
#pragma unroll
  for (int c = 0; c < 4; ++c) K3.v[c] = T(-1) * p[3].v[c] + T(-1) * p[4].v[c];
  R4<T> K4;
#pragma unroll
  for (int c = 0; c < 4; ++c) K4.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[3].v[c] + T(-1) * p[5].v[c];
  R4<T> K5;
#pragma unroll
  for (int c = 0; c < 4; ++c) K5.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[3].v[c];
  R4<T> K6;
#pragma unroll
  for (int c = 0; c < 4; ++c) K6.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[3].v[c] + T(-1) * p[4].v[c];
  R4<T> K7;
#pragma unroll
  for (int c = 0; c < 4; ++c) K7.v[c] = T(1) * p[0].v[c] + T(-1) * p[5].v[c];
  R4<T> K8;
#pragma unroll
  for (int c = 0; c < 4; ++c) K8.v[c] = T(1) * p[0].v[c] + T(-1) * p[4].v[c] + T(-1) * p[5].v[c];
  R4<T> K9;
#pragma unroll
  for (int c = 0; c < 4; ++c) K9.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[4].v[c] + T(-1) * p[5].v[c];
  R4<T> K10;
#pragma unroll
  for (int c = 0; c < 4; ++c) K10.v[c] = T(1) * p[0].v[c] + T(-1) * p[4].v[c];
  R4<T> K11;
#pragma unroll
  for (int c = 0; c < 4; ++c) K11.v[c] = T(-1) * p[1].v[c] + T(1) * p[4].v[c];
  R4<T> K12;
#pragma unroll
  for (int c = 0; c < 4; ++c) K12.v[c] = T(-1) * p[1].v[c] + T(1) * p[4].v[c] + T(1) * p[5].v[c];
  R4<T> K13;
#pragma unroll
  for (int c = 0; c < 4; ++c) K13.v[c] = T(-1) * p[1].v[c] + T(1) * p[5].v[c];
  R4<T> K14;
#pragma unroll
  for (int c = 0; c < 4; ++c) K14.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[4].v[c];
  R4<T> K15;
#pragma unroll
  for (int c = 0; c < 4; ++c) K15.v[c] = T(1) * p[0].v[c] + T(1) * p[1].v[c] + T(-1) * p[5].v[c];
  R4<T> K16;
#pragma unroll
  for (int c = 0; c < 4; ++c) K16.v[c] = T(-1) * p[4].v[c];
  R4<T> K17;
#pragma unroll
  for (int c = 0; c < 4; ++c) K17.v[c] = T(-1) * p[5].v[c];
  R4<T> K18;
#pragma unroll
  for (int c = 0; c < 4; ++c) K18.v[c] = T(-1) * p[4].v[c] + T(-1) * p[5].v[c];
  const V4<T> w0 = vcur(V2, U1);
  const V4<T> w1 = gprop(w0, K0);
  const S4<T> w2 = apply(make_slash(E6), VTB);
  const S4<T> w3 = hprop_col(K1, mt, mw, w2);
  const S4<T> w4 = apply(make_slash(E5), w3);
  const S4<T> w5 = hprop_col(K2, mt, mw, w4);
  const S4<T> w6 = apply(make_slash(w1), w5);
  const S4<T> w7 = apply(make_slash(E5), VTB);
  const S4<T> w8 = hprop_col(K3, mt, mw, w7);
  const S4<T> w9 = apply(make_slash(E6), w8);
  const S4<T> w10 = hprop_col(K2, mt, mw, w9);
  const S4<T> w11 = apply(make_slash(w1), w10);
  const S4<T> w12 = apply(make_slash(w1), w3);
  const S4<T> w13 = hprop_col(K4, mt, mw, w12);
  const S4<T> w14 = apply(make_slash(E5), w13);
  const S4<T> w15 = apply(make_slash(w1), VTB);
  const S4<T> w16 = hprop_col(K5, mt, mw, w15);
  const S4<T> w17 = apply(make_slash(E6), w16);
  const S4<T> w18 = hprop_col(K4, mt, mw, w17);
  const S4<T> w19 = apply(make_slash(E5), w18);
  const S4<T> w20 = apply(make_slash(w1), w8);
  const S4<T> w21 = hprop_col(K6, mt, mw, w20);
  const S4<T> w22 = apply(make_slash(E6), w21);
  const S4<T> w23 = apply(make_slash(E5), w16);
  const S4<T> w24 = hprop_col(K6, mt, mw, w23);
  const S4<T> w25 = apply(make_slash(E6), w24);
  const S4<T> w26 = apply(make_slash(E6), U1);
  const S4<T> w27 = lprop_col(K7, w26);
  const S4<T> w28 = apply(make_slash(E5), w27);
  const S4<T> w29 = lprop_col(K8, w28);
  const V4<T> w30 = vcur(V2, w29);
  const V4<T> w31 = gprop(w30, K9);
  const S4<T> w32 = apply(make_slash(w31), VTB);
  const S4<T> w33 = apply(make_slash(E5), U1);
  const S4<T> w34 = lprop_col(K10, w33);
  const S4<T> w35 = apply(make_slash(E6), w34);
  const S4<T> w36 = lprop_col(K8, w35);
  const V4<T> w37 = vcur(V2, w36);
  const V4<T> w38 = gprop(w37, K9);
  const S4<T> w39 = apply(make_slash(w38), VTB);
  const S4<T> w40 = slash_row(V2, E5);
  const S4<T> w41 = lprop_row(w40, K11);
  const V4<T> w42 = vcur(w41, w27);
  const V4<T> w43 = gprop(w42, K9);
  const S4<T> w44 = apply(make_slash(w43), VTB);
  const S4<T> w45 = slash_row(w41, E6);
  const S4<T> w46 = lprop_row(w45, K12);
  const V4<T> w47 = vcur(w46, U1);
  const V4<T> w48 = gprop(w47, K9);
  const S4<T> w49 = apply(make_slash(w48), VTB);
  const S4<T> w50 = slash_row(V2, E6);
  const S4<T> w51 = lprop_row(w50, K13);
  const V4<T> w52 = vcur(w51, w34);
  const V4<T> w53 = gprop(w52, K9);
  const S4<T> w54 = apply(make_slash(w53), VTB);
  const S4<T> w55 = slash_row(w51, E5);
  const S4<T> w56 = lprop_row(w55, K12);
  const V4<T> w57 = vcur(w56, U1);
  const V4<T> w58 = gprop(w57, K9);
  const S4<T> w59 = apply(make_slash(w58), VTB);
  const V4<T> w60 = vcur(V2, w34);
  const V4<T> w61 = gprop(w60, K14);
  const S4<T> w62 = apply(make_slash(w61), w3);
  const S4<T> w63 = apply(make_slash(w61), VTB);
  const S4<T> w64 = hprop_col(K6, mt, mw, w63);
  const S4<T> w65 = apply(make_slash(E6), w64);
  const V4<T> w66 = vcur(w41, U1);
  const V4<T> w67 = gprop(w66, K14);
  const S4<T> w68 = apply(make_slash(w67), w3);
  const S4<T> w69 = apply(make_slash(w67), VTB);
  const S4<T> w70 = hprop_col(K6, mt, mw, w69);
  const S4<T> w71 = apply(make_slash(E6), w70);
  const V4<T> w72 = vcur(V2, w27);
  const V4<T> w73 = gprop(w72, K15);
  const S4<T> w74 = apply(make_slash(w73), w8);
  const S4<T> w75 = apply(make_slash(w73), VTB);
  const S4<T> w76 = hprop_col(K4, mt, mw, w75);
  const S4<T> w77 = apply(make_slash(E5), w76);
  const V4<T> w78 = vcur(w51, U1);
  const V4<T> w79 = gprop(w78, K15);
  const S4<T> w80 = apply(make_slash(w79), w8);
  const S4<T> w81 = apply(make_slash(w79), VTB);
  const S4<T> w82 = hprop_col(K4, mt, mw, w81);
  const S4<T> w83 = apply(make_slash(E5), w82);
  const V4<T> w84 = vvv(w73, K15, E5, K16);
  const V4<T> w85 = gprop(w84, K9);
  const S4<T> w86 = apply(make_slash(w85), VTB);
  const V4<T> w87 = vvv(w79, K15, E5, K16);
  const V4<T> w88 = gprop(w87, K9);
  const S4<T> w89 = apply(make_slash(w88), VTB);
  const V4<T> w90 = vvv(w1, K0, E5, K16);
  const V4<T> w91 = gprop(w90, K14);
  const S4<T> w92 = apply(make_slash(w91), w3);
  const S4<T> w93 = apply(make_slash(w91), VTB);
  const S4<T> w94 = hprop_col(K6, mt, mw, w93);
  const S4<T> w95 = apply(make_slash(E6), w94);
  const V4<T> w96 = vvv(w61, K14, E6, K17);
  const V4<T> w97 = gprop(w96, K9);
  const S4<T> w98 = apply(make_slash(w97), VTB);
  const V4<T> w99 = vvv(w67, K14, E6, K17);
  const V4<T> w100 = gprop(w99, K9);
  const S4<T> w101 = apply(make_slash(w100), VTB);
  const V4<T> w102 = vvv(w1, K0, E6, K17);
  const V4<T> w103 = gprop(w102, K15);
  const S4<T> w104 = apply(make_slash(w103), w8);
  const S4<T> w105 = apply(make_slash(w103), VTB);
  const S4<T> w106 = hprop_col(K4, mt, mw, w105);
  const S4<T> w107 = apply(make_slash(E5), w106);
  const V4<T> w108 = vvv(w91, K14, E6, K17);
  const V4<T> w109 = gprop(w108, K9);
  const S4<T> w110 = apply(make_slash(w109), VTB);
  const V4<T> w111 = vvv(w103, K15, E5, K16);
  const V4<T> w112 = gprop(w111, K9);
  const S4<T> w113 = apply(make_slash(w112), VTB);
  const V4<T> w114 = v4_term<1>(w1, E5, E6);
  const V4<T> w115 = gprop(w114, K9);
  const S4<T> w116 = apply(make_slash(w115), VTB);
  const V4<T> w117 = v4_term<2>(w1, E5, E6);
  const V4<T> w118 = gprop(w117, K9);
  const S4<T> w119 = apply(make_slash(w118), VTB);
  const V4<T> w120 = v4_term<3>(w1, E5, E6);
  const V4<T> w121 = gprop(w120, K9);
  const S4<T> w122 = apply(make_slash(w121), VTB);
  const V4<T> w123 = vvv(E5, K16, E6, K17);
  const V4<T> w124 = gprop(w123, K18);
  const V4<T> w125 = vvv(w1, K0, w124, K18);
  const V4<T> w126 = gprop(w125, K9);
  const S4<T> w127 = apply(make_slash(w126), VTB);
  const S4<T> w128 = apply(make_slash(w124), U1);
  const S4<T> w129 = lprop_col(K8, w128);
  const V4<T> w130 = vcur(V2, w129);
  const V4<T> w131 = gprop(w130, K9);
  const S4<T> w132 = apply(make_slash(w131), VTB);
  const S4<T> w133 = slash_row(V2, w124);
  const S4<T> w134 = lprop_row(w133, K12);
  const V4<T> w135 = vcur(w134, U1);
  const V4<T> w136 = gprop(w135, K9);
  const S4<T> w137 = apply(make_slash(w136), VTB);
  const S4<T> w138 = apply(make_slash(w124), VTB);
  const S4<T> w139 = hprop_col(K2, mt, mw, w138);
  const S4<T> w140 = apply(make_slash(w1), w139);
  const S4<T> w141 = apply(make_slash(w124), w16);
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int b = 0; b < 12; ++b) J[h][b] = {T(0), T(0)};
  // diagram 0: light ['B'] bridge [] heavy ['B', 5, 6]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w6);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][10] = rfma(T(-0.16666666666666666), times_i(a), J[h][10]);
  }
  // diagram 1: light ['B'] bridge [] heavy ['B', 6, 5]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w11);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][11] = rfma(T(-0.16666666666666666), times_i(a), J[h][11]);
  }
  // diagram 2: light ['B'] bridge [] heavy [5, 'B', 6]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w14);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][10] = rfma(T(-0.16666666666666666), times_i(a), J[h][10]);
  }
  // diagram 3: light ['B'] bridge [] heavy [5, 6, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w19);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][10] = rfma(T(-0.16666666666666666), times_i(a), J[h][10]);
  }
  // diagram 4: light ['B'] bridge [] heavy [6, 'B', 5]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w22);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][11] = rfma(T(-0.16666666666666666), times_i(a), J[h][11]);
  }
  // diagram 5: light ['B'] bridge [] heavy [6, 5, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w25);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
    J[h][11] = rfma(T(-0.16666666666666666), times_i(a), J[h][11]);
  }
  // diagram 6: light ['B', 5, 6] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w32);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][6] = rfma(T(-0.16666666666666666), times_i(a), J[h][6]);
  }
  // diagram 7: light ['B', 6, 5] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w39);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
    J[h][7] = rfma(T(-0.16666666666666666), times_i(a), J[h][7]);
  }
  // diagram 8: light [5, 'B', 6] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w44);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][6] = rfma(T(-0.16666666666666666), times_i(a), J[h][6]);
  }
  // diagram 9: light [5, 6, 'B'] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w49);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][6] = rfma(T(-0.16666666666666666), times_i(a), J[h][6]);
  }
  // diagram 10: light [6, 'B', 5] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w54);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][7] = rfma(T(-0.16666666666666666), times_i(a), J[h][7]);
  }
  // diagram 11: light [6, 5, 'B'] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w59);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][7] = rfma(T(-0.16666666666666666), times_i(a), J[h][7]);
  }
  // diagram 12: light ['B', 5] bridge [] heavy ['B', 6]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w62);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][9] = rfma(T(-0.16666666666666666), times_i(a), J[h][9]);
  }
  // diagram 13: light ['B', 5] bridge [] heavy [6, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w65);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
    J[h][9] = rfma(T(-0.16666666666666666), times_i(a), J[h][9]);
  }
  // diagram 14: light [5, 'B'] bridge [] heavy ['B', 6]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w68);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][9] = rfma(T(-0.16666666666666666), times_i(a), J[h][9]);
  }
  // diagram 15: light [5, 'B'] bridge [] heavy [6, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w71);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][9] = rfma(T(-0.16666666666666666), times_i(a), J[h][9]);
  }
  // diagram 16: light ['B', 6] bridge [] heavy ['B', 5]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w74);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][8] = rfma(T(-0.16666666666666666), times_i(a), J[h][8]);
  }
  // diagram 17: light ['B', 6] bridge [] heavy [5, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w77);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][8] = rfma(T(-0.16666666666666666), times_i(a), J[h][8]);
  }
  // diagram 18: light [6, 'B'] bridge [] heavy ['B', 5]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w80);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][8] = rfma(T(-0.16666666666666666), times_i(a), J[h][8]);
  }
  // diagram 19: light [6, 'B'] bridge [] heavy [5, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w83);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][8] = rfma(T(-0.16666666666666666), times_i(a), J[h][8]);
  }
  // diagram 20: light ['B', 6] bridge [('v3', 5)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w86);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][4] = rfma(T(-0.5), times_i(a), J[h][4]);
  }
  // diagram 21: light [6, 'B'] bridge [('v3', 5)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w89);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
  }
  // diagram 22: light ['B'] bridge [('v3', 5)] heavy ['B', 6]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w92);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
  }
  // diagram 23: light ['B'] bridge [('v3', 5)] heavy [6, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w95);
    J[h][3] = rfma(T(0.5), times_i(a), J[h][3]);
    J[h][5] = rfma(T(-0.5), times_i(a), J[h][5]);
  }
  // diagram 24: light ['B', 5] bridge [('v3', 6)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w98);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][5] = rfma(T(-0.5), times_i(a), J[h][5]);
  }
  // diagram 25: light [5, 'B'] bridge [('v3', 6)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w101);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
  }
  // diagram 26: light ['B'] bridge [('v3', 6)] heavy ['B', 5]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w104);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
  }
  // diagram 27: light ['B'] bridge [('v3', 6)] heavy [5, 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w107);
    J[h][2] = rfma(T(0.5), times_i(a), J[h][2]);
    J[h][4] = rfma(T(-0.5), times_i(a), J[h][4]);
  }
  // diagram 28: light ['B'] bridge [('v3', 5), ('v3', 6)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w110);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
  }
  // diagram 29: light ['B'] bridge [('v3', 6), ('v3', 5)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w113);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
  }
  // diagram 30: light ['B'] bridge [('v4', 1)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w116);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
  }
  // diagram 31: light ['B'] bridge [('v4', 2)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w119);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][2] = rfma(T(-0.5), times_i(a), J[h][2]);
    J[h][3] = rfma(T(-0.5), times_i(a), J[h][3]);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
  }
  // diagram 32: light ['B'] bridge [('v4', 3)] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w122);
    J[h][0] = rfma(T(-0.5), times_i(a), J[h][0]);
    J[h][1] = rfma(T(0.5), times_i(a), J[h][1]);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][5] = rfma(T(-0.5), times_i(a), J[h][5]);
  }
  // diagram 33: light ['B'] bridge [('v3', 'G')] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w127);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][1] = rfma(T(-0.5), times_i(a), J[h][1]);
    J[h][4] = rfma(T(-0.5), times_i(a), J[h][4]);
    J[h][5] = rfma(T(0.5), times_i(a), J[h][5]);
  }
  // diagram 34: light ['B', 'G'] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w132);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][5] = rfma(T(-0.5), times_i(a), J[h][5]);
    J[h][6] = rfma(T(-0.16666666666666666), times_i(a), J[h][6]);
    J[h][7] = rfma(T(0.16666666666666666), times_i(a), J[h][7]);
  }
  // diagram 35: light ['G', 'B'] bridge [] heavy ['B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w137);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][1] = rfma(T(-0.5), times_i(a), J[h][1]);
    J[h][6] = rfma(T(-0.16666666666666666), times_i(a), J[h][6]);
    J[h][7] = rfma(T(0.16666666666666666), times_i(a), J[h][7]);
  }
  // diagram 36: light ['B'] bridge [] heavy ['B', 'G']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w140);
    J[h][0] = rfma(T(0.5), times_i(a), J[h][0]);
    J[h][1] = rfma(T(-0.5), times_i(a), J[h][1]);
    J[h][10] = rfma(T(-0.16666666666666666), times_i(a), J[h][10]);
    J[h][11] = rfma(T(0.16666666666666666), times_i(a), J[h][11]);
  }
  // diagram 37: light ['B'] bridge [] heavy ['G', 'B']
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cplx<T> a = rowdot(UB3[h], w141);
    J[h][4] = rfma(T(0.5), times_i(a), J[h][4]);
    J[h][5] = rfma(T(-0.5), times_i(a), J[h][5]);
    J[h][10] = rfma(T(-0.16666666666666666), times_i(a), J[h][10]);
    J[h][11] = rfma(T(0.16666666666666666), times_i(a), J[h][11]);
  }
}
// J^dagger (D C) J over the 12 colour structures (D = 3)
template <typename T>
__device__ __forceinline__ T uux_colour_form(const cplx<T> (&J)[12]) {
  T s = T(0);
  { cplx<T> y = T(24.0) * J[0];
    y = rfma(T(-6.0), J[1], y);
    y = rfma(T(6.0), J[4], y);
    y = rfma(T(6.0), J[5], y);
    y = rfma(T(16.0), J[6], y);
    y = rfma(T(-2.0), J[7], y);
    y = rfma(T(-2.0), J[8], y);
    y = rfma(T(16.0), J[9], y);
    y = rfma(T(16.0), J[10], y);
    y = rfma(T(-2.0), J[11], y);
    s = fma(J[0].r, y.r, fma(J[0].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[1];
    y = rfma(T(6.0), J[4], y);
    y = rfma(T(6.0), J[5], y);
    y = rfma(T(-2.0), J[6], y);
    y = rfma(T(16.0), J[7], y);
    y = rfma(T(16.0), J[8], y);
    y = rfma(T(-2.0), J[9], y);
    y = rfma(T(-2.0), J[10], y);
    y = rfma(T(16.0), J[11], y);
    s = fma(J[1].r, y.r, fma(J[1].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[2];
    y = rfma(T(6.0), J[3], y);
    y = rfma(T(-2.0), J[6], y);
    y = rfma(T(16.0), J[7], y);
    y = rfma(T(16.0), J[8], y);
    y = rfma(T(16.0), J[9], y);
    y = rfma(T(16.0), J[10], y);
    y = rfma(T(-2.0), J[11], y);
    s = fma(J[2].r, y.r, fma(J[2].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[3];
    y = rfma(T(16.0), J[6], y);
    y = rfma(T(-2.0), J[7], y);
    y = rfma(T(16.0), J[8], y);
    y = rfma(T(16.0), J[9], y);
    y = rfma(T(-2.0), J[10], y);
    y = rfma(T(16.0), J[11], y);
    s = fma(J[3].r, y.r, fma(J[3].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[4];
    y = rfma(T(-6.0), J[5], y);
    y = rfma(T(16.0), J[6], y);
    y = rfma(T(-2.0), J[7], y);
    y = rfma(T(16.0), J[8], y);
    y = rfma(T(-2.0), J[9], y);
    y = rfma(T(16.0), J[10], y);
    y = rfma(T(-2.0), J[11], y);
    s = fma(J[4].r, y.r, fma(J[4].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[5];
    y = rfma(T(-2.0), J[6], y);
    y = rfma(T(16.0), J[7], y);
    y = rfma(T(-2.0), J[8], y);
    y = rfma(T(16.0), J[9], y);
    y = rfma(T(-2.0), J[10], y);
    y = rfma(T(16.0), J[11], y);
    s = fma(J[5].r, y.r, fma(J[5].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[6];
    y = rfma(T(-6.0), J[7], y);
    y = rfma(T(6.0), J[10], y);
    y = rfma(T(6.0), J[11], y);
    s = fma(J[6].r, y.r, fma(J[6].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[7];
    y = rfma(T(6.0), J[10], y);
    y = rfma(T(6.0), J[11], y);
    s = fma(J[7].r, y.r, fma(J[7].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[8];
    y = rfma(T(6.0), J[9], y);
    s = fma(J[8].r, y.r, fma(J[8].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[9];
    s = fma(J[9].r, y.r, fma(J[9].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[10];
    y = rfma(T(-6.0), J[11], y);
    s = fma(J[10].r, y.r, fma(J[10].i, y.i, s)); }
  { cplx<T> y = T(24.0) * J[11];
    s = fma(J[11].r, y.r, fma(J[11].i, y.i, s)); }
  return T(2) * s;
}
}  // namespace mf
