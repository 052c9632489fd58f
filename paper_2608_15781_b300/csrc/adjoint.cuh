// Discrete adjoint of one time step (FP32 storage, one lattice, column mode,
// reaction mode 0): reverse mode through a1..a10 for the gradient of the outlet
// conversion J = 1 - Phi_out / Phi_in (Phi = sum over a z plane of u_z C).
//
// Given lambda_{t+1} = dJ/df_{t+1} (every stored population, ghost slots
// included) and the state f_t, one reverse step produces lambda_t = dJ/df_t and
// adds the step's share of dJ/dtheta (per solid node) and dJ/du_in.  The
// forward quantities of step t (rho^N, wetted normals, solid extrapolations) are
// recomputed from f_t by the forward kernels before the reverse kernels run:
//
//   collide   per fluid node: local adjoint of a2, a7 - a10 and of the outlet
//             ghost (non-equilibrium extrapolation), then the transpose of a1
//             (streaming, bounce-back, ghosts) as a push: the adjoint of each
//             pulled population goes to the stored population it came from
//             -> lambda_t without its density term (below), n_bar,
//             |grad|_bar, H_bar, rho, and the inlet ghost's share of dJ/du_in
//   curv      per interface node: transpose of the curvature stencil a6 -> n_bar
//   nsolid    per boundary solid: transpose of the solid-normal average -> n_bar
//   normal    per fluid node: transpose of a5 (wetting) and a4 (normalisation,
//             gradient stencil) -> rho^N_bar, theta_bar
//   csolid    per boundary solid: transpose of the solid-colour average a3
//   coef      per fluid node: d rho^N / d f coefficients times rho^N_bar, and
//             their share of dJ/du_in on plane 0
//
// A stored population of f_t enters the step through the node y that pulls it:
// through y's collision (the push above) and through rho^N(y) (a4).  The second
// term, coef(y), is known only after the stencil transposes, so lambda is kept
// without it and the collide kernel of the next reverse step adds coef(y) as it
// reads lambda_{t+1}; k_adj_finish adds it to lambda_0.  Each stored population
// is pulled by exactly one node or by none (it leaves the column): the push needs
// no atomics, and the owner of a population that leaves writes its zero.
//
// Branch decisions (the 1e-5 / 1e-6 thresholds, the n_+ / n_- choice, the
// reaction clamps) are those of the forward values, i.e. frozen.  Stencil
// transposes scatter with atomics (FP32 for per-step fields, FP64 for the
// gradients accumulated over all steps).
#pragma once

#include "compact.cuh"

namespace cglbm {

// adjoint of back_transform: bt_bar[0..17] -> u_bar, k5_bar..k9_bar (accumulated)
__device__ __forceinline__ void back_transform_adj(float ux, float uy, float uz, float k5, float k6, float k7,
                                                   float k8, float k9, const float (&bb)[Q], float &uxb,
                                                   float &uyb, float &uzb, float (&kb)[5]) {
  const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  {  // rows 0, 1
    const float A = ux2 - uy2 - uz2 + 1.0f;
    const float P = k5 * (1.0f / 3.0f) + k6 * (1.0f / 6.0f);
    const float R = uy * k7 + uz * k8;
    const float Ab = (bb[0] + bb[1]) * P;
    const float Pb = bb[0] * (A + ux) + bb[1] * (A - ux);
    const float Rb = -bb[0] * (2.0f * ux + 1.0f) - bb[1] * (2.0f * ux - 1.0f);
    uxb += bb[0] * (P - 2.0f * R) - bb[1] * (P + 2.0f * R) + 2.0f * ux * Ab;
    uyb += -2.0f * uy * Ab + k7 * Rb;
    uzb += -2.0f * uz * Ab + k8 * Rb;
    kb[0] += Pb * (1.0f / 3.0f);
    kb[1] += Pb * (1.0f / 6.0f);
    kb[2] += uy * Rb;
    kb[3] += uz * Rb;
  }
  {  // rows 2, 3
    const float B = ux2 - uy2 + uz2 - 1.0f;
    const float P = (k5 - k6) * (1.0f / 6.0f);
    const float R = ux * k7 + uz * k9;
    const float Bb = (bb[2] + bb[3]) * P;
    const float Pb = bb[2] * (B - uy) + bb[3] * (B + uy);
    const float Rb = -bb[2] * (2.0f * uy + 1.0f) - bb[3] * (2.0f * uy - 1.0f);
    uyb += -bb[2] * (P + 2.0f * R) + bb[3] * (P - 2.0f * R) - 2.0f * uy * Bb;
    uxb += 2.0f * ux * Bb + k7 * Rb;
    uzb += 2.0f * uz * Bb + k9 * Rb;
    kb[0] += Pb * (1.0f / 6.0f);
    kb[1] -= Pb * (1.0f / 6.0f);
    kb[2] += ux * Rb;
    kb[4] += uz * Rb;
  }
  {  // rows 4, 5
    const float Cc = ux2 + uy2 - uz2 - 1.0f;
    const float P = k5 * (1.0f / 6.0f) + k6 * (1.0f / 3.0f);
    const float R = ux * k8 + uy * k9;
    const float Cb = (bb[4] + bb[5]) * P;
    const float Pb = bb[4] * (Cc - uz) + bb[5] * (Cc + uz);
    const float Rb = -bb[4] * (2.0f * uz + 1.0f) - bb[5] * (2.0f * uz - 1.0f);
    uzb += -bb[4] * (P + 2.0f * R) + bb[5] * (P - 2.0f * R) - 2.0f * uz * Cb;
    uxb += 2.0f * ux * Cb + k8 * Rb;
    uyb += 2.0f * uy * Cb + k9 * Rb;
    kb[0] += Pb * (1.0f / 6.0f);
    kb[1] += Pb * (1.0f / 3.0f);
    kb[3] += ux * Rb;
    kb[4] += uy * Rb;
  }
  constexpr float T12 = 1.0f / 12.0f;
  {  // rows c = (a, b, 0)
    const int ia[4] = {6, 7, 10, 11};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CX[i], b = (float)CY[i], s = bb[i] * T12;
      kb[0] += s * (-ux2 - a * ux + 2.0f * uy2 + 2.0f * b * uy);
      kb[1] += s * (ux2 + a * ux + uy2 + b * uy);
      kb[2] += s * (12.0f * ux * uy + 6.0f * b * ux + 6.0f * a * uy + 3.0f * a * b);
      uxb += s * (k5 * (-2.0f * ux - a) + k6 * (2.0f * ux + a) + k7 * (12.0f * uy + 6.0f * b));
      uyb += s * (k5 * (4.0f * uy + 2.0f * b) + k6 * (2.0f * uy + b) + k7 * (12.0f * ux + 6.0f * a));
    }
  }
  {  // rows c = (a, 0, b)
    const int ia[4] = {8, 9, 12, 13};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CX[i], b = (float)CZ[i], s = bb[i] * T12;
      kb[0] += s * (-ux2 - a * ux + 2.0f * uz2 + 2.0f * b * uz);
      kb[1] += s * (-2.0f * ux2 - 2.0f * a * ux + uz2 + b * uz);
      kb[3] += s * (12.0f * ux * uz + 6.0f * b * ux + 6.0f * a * uz + 3.0f * a * b);
      uxb += s * (k5 * (-2.0f * ux - a) + k6 * (-4.0f * ux - 2.0f * a) + k8 * (12.0f * uz + 6.0f * b));
      uzb += s * (k5 * (4.0f * uz + 2.0f * b) + k6 * (2.0f * uz + b) + k8 * (12.0f * ux + 6.0f * a));
    }
  }
  {  // rows c = (0, a, b)
    const int ia[4] = {14, 15, 16, 17};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CY[i], b = (float)CZ[i], s = bb[i] * T12;
      kb[0] += s * (-uy2 - a * uy - uz2 - b * uz);
      kb[1] += s * (-2.0f * uy2 - 2.0f * a * uy + uz2 + b * uz);
      kb[4] += s * (12.0f * uy * uz + 6.0f * b * uy + 6.0f * a * uz + 3.0f * a * b);
      uyb += s * (k5 * (-2.0f * uy - a) + k6 * (-4.0f * uy - 2.0f * a) + k9 * (12.0f * uz + 6.0f * b));
      uzb += s * (k5 * (-2.0f * uz - b) + k6 * (2.0f * uz + b) + k9 * (12.0f * uy + 6.0f * a));
    }
  }
}

// adjoint of the outlet ghost (write_outlet_ghost_c) of a node of plane nz - 1:
// post-collision fr, fp; gr, gp = adjoint of the ghost's f^r, f^p (entries with
// c_z = -1 used).  Adds to lr, lp (adjoint of the post-collision populations).
__device__ __forceinline__ void outlet_ghost_adj(const float (&fr)[Q], const float (&fp)[Q], float rho_out,
                                                 const float (&gr)[Q], const float (&gp)[Q], float (&lr)[Q],
                                                 float (&lp)[Q]) {
  float rho = 0.f, rr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float m = fr[i] + fp[i];
    rho += m;
    rr += fr[i];
    jx += CX[i] * m;
    jy += CY[i] * m;
    jz += CZ[i] * m;
  }
  const float inv = 1.0f / rho;
  const float vx = jx * inv, vy = jy * inv, vz = jz * inv;
  const float vv = vx * vx + vy * vy + vz * vz;
  const float psi = rr * inv;
  float psib = 0.f, rhob = 0.f, vxb = 0.f, vyb = 0.f, vzb = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != -1) continue;
    lr[i] += gr[i];
    lp[i] += gp[i];
    const float cu = CX[i] * vx + CY[i] * vy + CZ[i] * vz;
    const float E = W[i] * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * vv);
    const float corr = (rho_out - rho) * E;
    const float cb = psi * gr[i] + (1.0f - psi) * gp[i];
    psib += corr * (gr[i] - gp[i]);
    rhob -= cb * E;
    const float s = cb * W[i] * (rho_out - rho);
    const float t = s * (3.0f + 9.0f * cu);
    vxb += t * CX[i] - 3.0f * s * vx;
    vyb += t * CY[i] - 3.0f * s * vy;
    vzb += t * CZ[i] - 3.0f * s * vz;
  }
  const float rrb = psib * inv;
  rhob -= psib * psi * inv;
  const float jxb = vxb * inv, jyb = vyb * inv, jzb = vzb * inv;
  rhob -= (vxb * vx + vyb * vy + vzb * vz) * inv;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float mb = jxb * CX[i] + jyb * CY[i] + jzb * CZ[i] + rhob;
    lr[i] += mb + rrb;
    lp[i] += mb;
  }
}

// adjoint of collide_node (reaction mode 0).  In: pulled fr, fp, g; nme, H; lr,
// lp, lg = adjoint of the post-collision f^r*, f^p*, g*.  Out: lr, lp, lg =
// adjoint of the pulled populations; nb = adjoint of n, wb of |grad rho^N|, Hb
// of H.  Returns rho^m.
__device__ __forceinline__ float collide_node_adj(const StepParams &P, uint32_t lk, const float (&fr)[Q],
                                                  const float (&fp)[Q], const float (&g)[Q7], const float4 nme,
                                                  float H, float (&lr)[Q], float (&lp)[Q], float (&lg)[Q7],
                                                  float &nbx, float &nby, float &nbz, float &wb, float &Hb) {
  // forward recompute (same arithmetic as collide_node)
  float rr = 0.f, rp = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rr += fr[i];
    rp += fp[i];
    const float m = fr[i] + fp[i];
    if (CX[i]) jx += CX[i] * m;
    if (CY[i]) jy += CY[i] * m;
    if (CZ[i]) jz += CZ[i] * m;
    if (CX[i]) pxx += m;
    if (CY[i]) pyy += m;
    if (CZ[i]) pzz += m;
    if (CX[i] && CY[i]) pxy += CX[i] * CY[i] * m;
    if (CX[i] && CZ[i]) pxz += CX[i] * CZ[i] * m;
    if (CY[i] && CZ[i]) pyz += CY[i] * CZ[i] * m;
  }
  const float rho = rr + rp;
  const float inv_rho = 1.0f / rho;
  const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
  const float fs = P.half_sigma * H * nme.w * inv_rho;
  const float dux = fs * nme.x + P.ax, duy = fs * nme.y + P.ay, duz = fs * nme.z + P.az;
  const float om = P.omega_cm;
  const float k5 = om * ((pxx - pyy) - rho * (ux * ux - uy * uy));
  const float k6 = om * ((pyy - pzz) - rho * (uy * uy - uz * uz));
  const float k7 = om * (pxy - rho * ux * uy);
  const float k8 = om * (pxz - rho * ux * uz);
  const float k9 = om * (pyz - rho * uy * uz);
  float bt[Q];
  back_transform(ux, uy, uz, k5, k6, k7, k8, k9, bt);
  const float vx = ux + dux, vy = uy + duy, vz = uz + duz;
  const float vv = vx * vx + vy * vy + vz * vz;
  const float psi = rr * inv_rho;
  const float knn = P.k_rate * (float)((lk >> NN_SHIFT) & 7u);
  float conc = 0.f;
#pragma unroll
  for (int j = 0; j < Q7; ++j) conc += g[j];
  int br = 0;   // active reaction branch: 0 none, 1 k NN C psi, 2 C, 3 rho^r
  if (lk & BIT_REACTIVE) {
    const float a = knn * conc * psi;
    const float d1 = fminf(a, conc);
    const int b1 = a <= conc ? 1 : 2;
    const float d = fminf(d1, rr);
    br = d1 <= rr ? b1 : 3;
    if (d < 0.f) br = 0;
  }
  const float Brec = P.beta * rr * rp * inv_rho;
  float fms[Q];
  {
    float msum = 0.f;
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
      fms[i] = feq19(i, rho, vx, vy, vz, vv) + bt[i];
      msum += fms[i];
    }
    fms[Q - 1] = rho - msum;
  }
  const float wx = ux + 0.5f * dux, wy = uy + 0.5f * duy, wz = uz + 0.5f * duz;

  // reverse: recolouring + reaction transfer
  float FMb[Q];
  float psib = 0.f, Bb = 0.f, deltab = 0.f;
  nbx = nby = nbz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float Rb = lr[i] - lp[i];
    FMb[i] = lp[i] + psi * Rb;
    psib += fms[i] * Rb;
    const float cn = (CX[i] * nme.x + CY[i] * nme.y + CZ[i] * nme.z) * INVNORM[i];
    Bb += W[i] * cn * Rb;
    const float t = W[i] * Brec * Rb * INVNORM[i];
    nbx += t * CX[i];
    nby += t * CY[i];
    nbz += t * CZ[i];
    deltab -= W[i] * Rb;
  }
  // D3Q7 BGK
  float Cb = 0.f, wxb = 0.f, wyb = 0.f, wzb = 0.f;
  const float itg = P.inv_tau_g;
#pragma unroll
  for (int j = 0; j < Q7; ++j) {
    const int dd = GDIR[j];
    deltab -= W7[j] * lg[j];
    const float geqb = lg[j] * itg;
    const float cw = CX[dd] * wx + CY[dd] * wy + CZ[dd] * wz;
    Cb += geqb * W7[j] * (1.0f + 4.0f * cw);
    const float t = geqb * W7[j] * conc * 4.0f;
    wxb += t * CX[dd];
    wyb += t * CY[dd];
    wzb += t * CZ[dd];
    lg[j] *= 1.0f - itg;
  }
  float uxb = wxb, uyb = wyb, uzb = wzb;
  float duxb = 0.5f * wxb, duyb = 0.5f * wyb, duzb = 0.5f * wzb;
  // rest population from mass conservation, equilibrium part
  float rhob = FMb[Q - 1];
  float vxb = 0.f, vyb = 0.f, vzb = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const float f = FMb[i] - FMb[Q - 1];
    FMb[i] = f;   // now the adjoint of bt[i]
    const float cu = CX[i] * vx + CY[i] * vy + CZ[i] * vz;
    rhob += f * W[i] * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * vv);
    const float s = f * W[i] * rho;
    const float t = s * (3.0f + 9.0f * cu);
    vxb += t * CX[i] - 3.0f * s * vx;
    vyb += t * CY[i] - 3.0f * s * vy;
    vzb += t * CZ[i] - 3.0f * s * vz;
  }
  // reaction amount (frozen branch)
  float rrb = 0.f, rpb = 0.f;
  if (br == 1) {
    Cb += deltab * knn * psi;
    psib += deltab * knn * conc;
  } else if (br == 2) {
    Cb += deltab;
  } else if (br == 3) {
    rrb += deltab;
  }
  // recolouring amplitude and colour ratio
  rrb += Bb * P.beta * rp * inv_rho;
  rpb += Bb * P.beta * rr * inv_rho;
  rhob -= Bb * Brec * inv_rho;
  rrb += psib * inv_rho;
  rhob -= psib * psi * inv_rho;
#pragma unroll
  for (int j = 0; j < Q7; ++j) lg[j] += Cb;
  // v = u + du
  uxb += vxb;
  uyb += vyb;
  uzb += vzb;
  duxb += vxb;
  duyb += vyb;
  duzb += vzb;
  // central moments
  float kb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  back_transform_adj(ux, uy, uz, k5, k6, k7, k8, k9, FMb, uxb, uyb, uzb, kb);
  const float pxxb = om * kb[0], pyyb = om * (kb[1] - kb[0]), pzzb = -om * kb[1];
  const float pxyb = om * kb[2], pxzb = om * kb[3], pyzb = om * kb[4];
  rhob -= om * (kb[0] * (ux * ux - uy * uy) + kb[1] * (uy * uy - uz * uz) + kb[2] * ux * uy + kb[3] * ux * uz +
                kb[4] * uy * uz);
  uxb -= om * rho * (2.0f * ux * kb[0] + uy * kb[2] + uz * kb[3]);
  uyb -= om * rho * (-2.0f * uy * kb[0] + 2.0f * uy * kb[1] + ux * kb[2] + uz * kb[4]);
  uzb -= om * rho * (-2.0f * uz * kb[1] + ux * kb[3] + uy * kb[4]);
  // du = fs n + a, fs = (sigma/2) H |grad| / rho
  const float fsb = duxb * nme.x + duyb * nme.y + duzb * nme.z;
  nbx += fs * duxb;
  nby += fs * duyb;
  nbz += fs * duzb;
  Hb = fsb * P.half_sigma * nme.w * inv_rho;
  wb = fsb * P.half_sigma * H * inv_rho;
  rhob -= fsb * fs * inv_rho;
  // u = j / rho
  const float jxb = uxb * inv_rho, jyb = uyb * inv_rho, jzb = uzb * inv_rho;
  rhob -= (uxb * ux + uyb * uy + uzb * uz) * inv_rho;
  rrb += rhob;
  rpb += rhob;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float mb = jxb * CX[i] + jyb * CY[i] + jzb * CZ[i];
    if (CX[i]) mb += pxxb;
    if (CY[i]) mb += pyyb;
    if (CZ[i]) mb += pzzb;
    if (CX[i] && CY[i]) mb += CX[i] * CY[i] * pxyb;
    if (CX[i] && CZ[i]) mb += CX[i] * CZ[i] * pxzb;
    if (CY[i] && CZ[i]) mb += CY[i] * CZ[i] * pyzb;
    lr[i] = mb + rrb;
    lp[i] = mb + rpb;
  }
  return rho;
}

// dJ/df of the objective at the stored state f: a_in = dJ/dPhi_in on plane 0,
// a_out = dJ/dPhi_out on plane nz - 1, Phi = sum u_z C with u_z = j_z / rho.
__global__ void k_adj_seed(Slots S, const __grid_constant__ Inst I, const float *__restrict__ f, float a_in,
                           float a_out, float *__restrict__ lam) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const unsigned ns = (unsigned)S.ns;
  const uint32_t pk = S.node[t];
  float a = 0.f;
  int x = 0, y = 0, z = -1;
  if (pk != kNoNode) {
    unpack(pk, x, y, z);
    if (z == 0) a = a_in;
    if (z == I.L.nz - 1) a = a_out;
  }
  if (a == 0.f) {
    for (int p = 0; p < NPOP; ++p) lam[(unsigned)p * ns + t] = 0.f;
    return;
  }
  float rho = 0.f, jz = 0.f, cc = 0.f;
  for (int i = 0; i < Q; ++i) {
    float fr, fp;
    Store<float>::ld2(f, ns, i, t, i, fr, fp);   // the forward state, in the slot layout
    const float m = fr + fp;
    rho += m;
    jz += CZ[i] * m;
  }
  for (int j = 0; j < Q7; ++j) cc += Store<float>::ld(f, ns, 2 * Q + j, t);
  const float inv = 1.0f / rho;
  for (int i = 0; i < Q; ++i) {
    const float v = a * cc * (CZ[i] * inv - jz * inv * inv);
    lam[(unsigned)i * ns + t] = v;
    lam[(unsigned)(Q + i) * ns + t] = v;
  }
  for (int j = 0; j < Q7; ++j) lam[(unsigned)(2 * Q + j) * ns + t] = a * jz * inv;
}

// collide: local adjoint at every fluid slot and the push of a1's transpose
// lam_in: lambda_{t+1} without its density terms, coef_in the coefficients of the
// reverse step t + 1 (zero for the objective's seed); lam_out: lambda_t without
// its density terms.
__global__ void __launch_bounds__(128, 3) k_adj_collide(Slots S, const __grid_constant__ Inst I,
                                                     const float *__restrict__ fin, const int *__restrict__ gidx,
                                                     const uint32_t *__restrict__ link,
                                                     const float4 *__restrict__ nrm, const float *__restrict__ Hs,
                                                     const float *__restrict__ lam, const float2 *__restrict__ coef_in,
                                                     float u_in, float c_in, float *__restrict__ lam_out,
                                                     float4 *__restrict__ nbar, float *__restrict__ hbar,
                                                     float *__restrict__ rho_out, double *__restrict__ uin_acc) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double du = 0.0;
  const uint32_t pk = t < (unsigned)S.nslots ? S.node[t] : kNoNode;
  if (pk != kNoNode) {
    int x, y, z;
    unpack(pk, x, y, z);
    const Lattice &L = I.L;
    StencilOffsets St;
    St.init(L, x, y, z);
    const unsigned node = St.own;
    const uint32_t lk = link[node];
    const float4 nme = nrm[node];
    // the curvature of the forward step: stored by the recompute's main kernel (Hs), or computed here
    float H;
    if (Hs)
      H = Hs[node];
    else
      H = nme.w >= GRAD_EPS ? curvature(nme, [&](int i) { return nrm[St.nb(CX[i], CY[i], CZ[i])]; }) : 0.f;
    PullOffsets O;
    O.init(L, x, y, z);
    int src[Q];
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) src[i] = __ldg(gidx + O.src(CX[i], CY[i], CZ[i]));
    src[Q - 1] = (int)t;
    const unsigned ns = (unsigned)S.ns;
    float fr[Q], fp[Q], g[Q7];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const bool bb = src[i] < 0;
      Store<float>::ld2(fin, ns, bb ? (unsigned)OPP[i] : (unsigned)i, bb ? t : (unsigned)src[i], i, fr[i], fp[i]);
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) {
      const int d = GDIR[j];
      const bool bb = src[d] < 0;
      g[j] = Store<float>::ld(fin, ns, 2 * Q + (bb ? GOPP[j] : j), bb ? t : (unsigned)src[d]);
    }
    // lambda_{t+1} of this slot's populations, each with the density term of the node
    // that pulls it: x + c_i when fluid, x itself when x + c_i is solid (bounce-back),
    // none when x + c_i leaves the column
    float lr[Q], lp[Q], lg[Q7];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      lr[i] = lam[(unsigned)i * ns + t];
      lp[i] = lam[(unsigned)(Q + i) * ns + t];
      const int zt = z + CZ[i];
      if (L.bc_z == 0 || (zt >= 0 && zt < L.nz)) {
        const bool solid = i < Q - 1 && ((lk >> OPP[i]) & 1u);   // x + c_i is the source of direction OPP[i]
        const float2 c2 = __ldg(coef_in + ((i == Q - 1 || solid) ? node : St.nb(CX[i], CY[i], CZ[i])));
        lr[i] += c2.x;
        lp[i] += c2.y;
      }
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) lg[j] = lam[(unsigned)(2 * Q + j) * ns + t];
    if (L.bc_z == 1 && z == L.nz - 1) {
      // the outlet ghost above this node is a function of its post-collision populations;
      // its population i (c_z = -1) is pulled by the fluid node x + (c_x, c_y, 0) of this plane
      const unsigned gs = (unsigned)(I.ghost + L.plane) + (unsigned)(y * L.nx + x);
      float sr[Q], sp[Q], sg[Q7], gr[Q], gp[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        sr[i] = fr[i];
        sp[i] = fp[i];
        gr[i] = 0.f;
        gp[i] = 0.f;
        if (CZ[i] == -1) {
          gr[i] = lam[(unsigned)i * ns + gs];
          gp[i] = lam[(unsigned)(Q + i) * ns + gs];
          const int xd = x + CX[i] < 0 ? L.nx - 1 : (x + CX[i] >= L.nx ? 0 : x + CX[i]);
          const int yd = y + CY[i] < 0 ? L.ny - 1 : (y + CY[i] >= L.ny ? 0 : y + CY[i]);
          const long long dn = ((long long)z * L.ny + yd) * L.nx + xd;
          if (!(link[dn] & BIT_SOLID)) {
            const float2 c2 = __ldg(coef_in + dn);
            gr[i] += c2.x;
            gp[i] += c2.y;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < Q7; ++j) sg[j] = g[j];
      collide_node(I.P, lk, sr, sp, sg, nme, H);
      outlet_ghost_adj(sr, sp, I.P.rho_out, gr, gp, lr, lp);
      lg[5] += lam[(unsigned)(2 * Q + 5) * ns + gs];
    }
    float nbx, nby, nbz, wb, Hb;
    const float rho = collide_node_adj(I.P, lk, fr, fp, g, nme, H, lr, lp, lg, nbx, nby, nbz, wb, Hb);
    // push: the adjoint of each pulled population to the population it was pulled from
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const bool bb = src[i] < 0;
      const unsigned s_ = bb ? t : (unsigned)src[i], pr = bb ? (unsigned)OPP[i] : (unsigned)i;
      lam_out[pr * ns + s_] = lr[i];
      lam_out[(Q + pr) * ns + s_] = lp[i];
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) {
      const int d = GDIR[j];
      const bool bb = src[d] < 0;
      lam_out[(unsigned)(2 * Q + (bb ? GOPP[j] : j)) * ns + (bb ? t : (unsigned)src[d])] = lg[j];
    }
    if (L.bc_z == 1) {
      // populations of this slot that leave the column: pulled by nobody, adjoint 0
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if ((z == 0 && CZ[i] == -1) || (z == L.nz - 1 && CZ[i] == 1)) {
          lam_out[(unsigned)i * ns + t] = 0.f;
          lam_out[(unsigned)(Q + i) * ns + t] = 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < Q7; ++j) {
        const int cz = CZ[GDIR[j]];
        if ((z == 0 && cz == -1) || (z == L.nz - 1 && cz == 1)) lam_out[(unsigned)(2 * Q + j) * ns + t] = 0.f;
      }
      // the inlet ghost's populations entering at plane 0: f^r_i = f^eq_i(1, u_in z)
      // (c_iz = 1), g_4 = w_4 c_in (1 + 4 u_in); here without their density terms (k_adj_coef)
      if (z == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (CZ[i] == 1) s += (double)lr[i] * (double)(W[i] * (3.0f + 6.0f * u_in));
        s += (double)lg[4] * (double)(4.0f * W7[4] * c_in);
        du = s;
      }
    }
    nbar[node] = make_float4(nbx, nby, nbz, wb);
    hbar[node] = nme.w >= GRAD_EPS ? Hb : 0.f;
    rho_out[node] = rho;
  }
  du = warp_sum(du);
  if ((threadIdx.x & 31) == 0 && du != 0.0) atomicAdd(uin_acc, du);
}

// curv: H = -sum_i 3 w_i (c_i - (n.c_i) n) . n(x + c_i); dH/dn = (D + D^T) n
__global__ void k_adj_curv(Slots S, const __grid_constant__ Inst I, const float4 *__restrict__ nrm,
                           const float *__restrict__ hbar, float4 *__restrict__ nbar) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const uint32_t pk = S.node[t];
  if (pk == kNoNode) return;
  int x, y, z;
  unpack(pk, x, y, z);
  StencilOffsets St;
  St.init(I.L, x, y, z);
  const unsigned node = St.own;
  const float4 nme = nrm[node];
  if (nme.w < GRAD_EPS) return;
  const float Hb = hbar[node];
  if (Hb == 0.f) return;
  float d[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  for (int i = 0; i < Q - 1; ++i) {
    const unsigned nb = St.nb(CX[i], CY[i], CZ[i]);
    const float4 v = nrm[nb];
    const float w3 = 3.0f * W[i];
    const float c[3] = {(float)CX[i], (float)CY[i], (float)CZ[i]};
    for (int a = 0; a < 3; ++a) {
      d[a][0] += w3 * c[a] * v.x;
      d[a][1] += w3 * c[a] * v.y;
      d[a][2] += w3 * c[a] * v.z;
    }
    const float cn = c[0] * nme.x + c[1] * nme.y + c[2] * nme.z;
    const float s = -w3 * Hb;
    atomicAdd(&nbar[nb], make_float4(s * (c[0] - cn * nme.x), s * (c[1] - cn * nme.y), s * (c[2] - cn * nme.z),
                                     0.f));
  }
  const float n3[3] = {nme.x, nme.y, nme.z};
  float o[3];
  for (int a = 0; a < 3; ++a) {
    o[a] = 0.f;
    for (int b = 0; b < 3; ++b) o[a] += (d[a][b] + d[b][a]) * n3[b];
  }
  atomicAdd(&nbar[node], make_float4(Hb * o[0], Hb * o[1], Hb * o[2], 0.f));
}

// nsolid: n(s) = A / |A|, A = sum_i w_i n(s + c_i) over fluid neighbours
__global__ void k_adj_nsolid(const __grid_constant__ Inst I, const uint32_t *__restrict__ list, int count,
                             const uint32_t *__restrict__ link, const float4 *__restrict__ nrm,
                             float4 *__restrict__ nbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int x, y, z;
  unpack(list[t], x, y, z);
  StencilOffsets St;
  St.init(I.L, x, y, z);
  const uint32_t lk = link[St.own];
  float ax = 0.f, ay = 0.f, az = 0.f;
  for (int i = 0; i < Q - 1; ++i) {
    if ((lk >> i) & 1u) {
      const float4 v = nrm[St.nb(CX[i], CY[i], CZ[i])];
      ax += W[i] * v.x;
      ay += W[i] * v.y;
      az += W[i] * v.z;
    }
  }
  const float m = sqrtf(ax * ax + ay * ay + az * az);
  if (m < GRAD_EPS) return;
  const float4 nb4 = nbar[St.own];
  const float inv = 1.0f / m;
  const float nx_ = ax * inv, ny_ = ay * inv, nz_ = az * inv;
  const float dn = nx_ * nb4.x + ny_ * nb4.y + nz_ * nb4.z;
  const float bx = (nb4.x - dn * nx_) * inv, by = (nb4.y - dn * ny_) * inv, bz = (nb4.z - dn * nz_) * inv;
  if (bx == 0.f && by == 0.f && bz == 0.f) return;
  for (int i = 0; i < Q - 1; ++i) {
    if ((lk >> i) & 1u) {
      atomicAdd(&nbar[St.nb(CX[i], CY[i], CZ[i])], make_float4(W[i] * bx, W[i] * by, W[i] * bz, 0.f));
    }
  }
}

// normal: transpose of a5 (wetting, frozen n_+/n_- choice) and a4; scatters
// rho^N_bar to the stencil and theta_bar (degrees) to the solid neighbours
__global__ void k_adj_normal(Slots S, const __grid_constant__ Inst I, const float *__restrict__ rhoN,
                             const uint32_t *__restrict__ link, const float4 *__restrict__ ns,
                             const float4 *__restrict__ nbar, float *__restrict__ rnbar,
                             double *__restrict__ thbar) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const uint32_t pk = S.node[t];
  if (pk == kNoNode) return;
  int x, y, z;
  unpack(pk, x, y, z);
  StencilOffsets St;
  St.init(I.L, x, y, z);
  const unsigned node = St.own;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  for (int i = 0; i < Q - 1; ++i) {
    const float v = 3.0f * W[i] * rhoN[St.nb(CX[i], CY[i], CZ[i])];
    gx += CX[i] * v;
    gy += CY[i] * v;
    gz += CZ[i] * v;
  }
  const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
  if (gm < GRAD_EPS) return;
  const float4 nb4 = nbar[node];
  const float inv = 1.0f / gm;
  const float n0 = gx * inv, n1 = gy * inv, n2 = gz * inv;
  float rx = nb4.x, ry = nb4.y, rz = nb4.z;   // adjoint of the unwetted normal
  const uint32_t lk = link[node];
  float thb = 0.f;
  if ((lk & BIT_WALL) && (lk & BIT_NS_OK)) {
    const float4 s = ns[node];
    const float c = s.x * n0 + s.y * n1 + s.z * n2;
    const float tx = n0 - c * s.x, ty = n1 - c * s.y, tz = n2 - c * s.z;
    const float st2 = tx * tx + ty * ty + tz * tz;
    if (st2 >= SIN2_EPS) {
      float sin_th, cos_th;
      sincosf(s.w, &sin_th, &cos_th);
      const float st = sqrtf(st2);
      const float a_s = sin_th * c / st, a_n = sin_th / st;
      const float px = (cos_th - a_s) * s.x + a_n * n0, py = (cos_th - a_s) * s.y + a_n * n1,
                  pz = (cos_th - a_s) * s.z + a_n * n2;
      const float mx = (cos_th + a_s) * s.x - a_n * n0, my = (cos_th + a_s) * s.y - a_n * n1,
                  mz = (cos_th + a_s) * s.z - a_n * n2;
      const float dp = (px - n0) * (px - n0) + (py - n1) * (py - n1) + (pz - n2) * (pz - n2);
      const float dm = (mx - n0) * (mx - n0) + (my - n1) * (my - n1) + (mz - n2) * (mz - n2);
      const float sg = dp <= dm ? 1.0f : -1.0f;
      // n_wet = A s + B n, A = cos - sg sin c / st, B = sg sin / st, st = sqrt(1 - c^2)
      const float B = sg * sin_th / st;
      const float st3 = st2 * st;
      const float dA = -sg * sin_th / st3, dB = sg * sin_th * c / st3;
      const float snb = s.x * nb4.x + s.y * nb4.y + s.z * nb4.z;
      const float nnb = n0 * nb4.x + n1 * nb4.y + n2 * nb4.z;
      const float cb = dA * snb + dB * nnb;
      rx = B * nb4.x + cb * s.x;
      ry = B * nb4.y + cb * s.y;
      rz = B * nb4.z + cb * s.z;
      thb = (-sin_th - sg * cos_th * c / st) * snb + (sg * cos_th / st) * nnb;   // per radian
    }
  }
  const float dr = n0 * rx + n1 * ry + n2 * rz;
  const float bx = (rx - dr * n0) * inv + nb4.w * n0;
  const float by = (ry - dr * n1) * inv + nb4.w * n1;
  const float bz = (rz - dr * n2) * inv + nb4.w * n2;
  for (int i = 0; i < Q - 1; ++i) {
    const float v = 3.0f * W[i] * (CX[i] * bx + CY[i] * by + CZ[i] * bz);
    if (v != 0.f) atomicAdd(&rnbar[St.nb(CX[i], CY[i], CZ[i])], v);
  }
  if (thb != 0.f) {
    float den = 0.f;
    for (int i = 0; i < Q - 1; ++i)
      if (link[St.nb(CX[i], CY[i], CZ[i])] & BIT_SOLID) den += W[i];
    const double scale = (double)thb * 0.017453292519943295 / (double)den;
    for (int i = 0; i < Q - 1; ++i) {
      const unsigned nb = St.nb(CX[i], CY[i], CZ[i]);
      if (link[nb] & BIT_SOLID) atomicAdd(&thbar[nb], scale * (double)W[i]);
    }
  }
}

// csolid: rho^N(s) = sum_i w_i rho^N(s + c_i) / sum_i w_i over fluid neighbours
__global__ void k_adj_csolid(const __grid_constant__ Inst I, const uint32_t *__restrict__ list, int count,
                             const uint32_t *__restrict__ link, float *__restrict__ rnbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int x, y, z;
  unpack(list[t], x, y, z);
  StencilOffsets St;
  St.init(I.L, x, y, z);
  const float rb = rnbar[St.own];
  if (rb == 0.f) return;
  const uint32_t lk = link[St.own];
  float den = 0.f;
  for (int i = 0; i < Q - 1; ++i)
    if ((lk >> i) & 1u) den += W[i];
  if (!(den > 0.f)) return;
  const float s = rb / den;
  for (int i = 0; i < Q - 1; ++i)
    if ((lk >> i) & 1u) atomicAdd(&rnbar[St.nb(CX[i], CY[i], CZ[i])], W[i] * s);
}

// coef: rho^N = (rho^r - rho^p) / rho  ->  d/d f^r_i = (1 - rho^N)/rho, d/d f^p_i = -(1 + rho^N)/rho
// On plane 0 of a column the pulled f^r_i with c_iz = 1 are the inlet ghost's, so their
// density terms add to dJ/du_in.
__global__ void k_adj_coef(Slots S, const __grid_constant__ Inst I, const float *__restrict__ rhoN,
                           const float *__restrict__ rho, const float *__restrict__ rnbar, float u_in,
                           float2 *__restrict__ coef, double *__restrict__ uin_acc) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double du = 0.0;
  const uint32_t pk = t < (unsigned)S.nslots ? S.node[t] : kNoNode;
  if (pk != kNoNode) {
    int x, y, z;
    unpack(pk, x, y, z);
    const long long node = nidx(I.L, x, y, z);
    const float rb = rnbar[node], r = rhoN[node], inv = 1.0f / rho[node];
    const float2 c2 = make_float2(rb * (1.0f - r) * inv, -rb * (1.0f + r) * inv);
    coef[node] = c2;
    if (I.L.bc_z == 1 && z == 0) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (CZ[i] == 1) du += (double)c2.x * (double)(W[i] * (3.0f + 6.0f * u_in));
    }
  }
  du = warp_sum(du);
  if ((threadIdx.x & 31) == 0 && du != 0.0) atomicAdd(uin_acc, du);
}

// lambda_0 with its density terms: every population of a fluid slot, and the outlet
// ghost's populations entering the column (read by k_adj_ghost0), gain coef of the
// node that pulls them (the same rule as the collide kernel's read of lambda_{t+1})
__global__ void k_adj_finish(Slots S, const __grid_constant__ Inst I, const uint32_t *__restrict__ link,
                             const float2 *__restrict__ coef, float *__restrict__ lam) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const Lattice &L = I.L;
  const unsigned ns = (unsigned)S.ns;
  const uint32_t pk = S.node[t];
  if (pk != kNoNode) {
    int x, y, z;
    unpack(pk, x, y, z);
    StencilOffsets St;
    St.init(L, x, y, z);
    const uint32_t lk = link[St.own];
    for (int i = 0; i < Q; ++i) {
      const int zt = z + CZ[i];
      if (L.bc_z == 1 && (zt < 0 || zt >= L.nz)) continue;
      const bool solid = i < Q - 1 && ((lk >> OPP[i]) & 1u);
      const float2 c2 = coef[(i == Q - 1 || solid) ? St.own : St.nb(CX[i], CY[i], CZ[i])];
      lam[(unsigned)i * ns + t] += c2.x;
      lam[(unsigned)(Q + i) * ns + t] += c2.y;
    }
    return;
  }
  if (L.bc_z != 1 || (long long)t < (long long)I.ghost + L.plane) return;   // inlet ghosts: not needed
  const long long r = (long long)t - I.ghost - L.plane;                       // outlet ghost (x, y, nz)
  const int y = (int)(r / L.nx), x = (int)(r % L.nx);
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != -1) continue;
    const int xd = (x + CX[i] + L.nx) % L.nx, yd = (y + CY[i] + L.ny) % L.ny;
    const long long dn = ((long long)(L.nz - 1) * L.ny + yd) * L.nx + xd;
    if (link[dn] & BIT_SOLID) continue;
    lam[(unsigned)i * ns + t] += coef[dn].x;
    lam[(unsigned)(Q + i) * ns + t] += coef[dn].y;
  }
}

// The outlet ghost of the start state is the extrapolation of its plane nz - 1:
// fold the ghost's adjoint into the adjoint of those stored populations.
__global__ void k_adj_ghost0(Slots S, const __grid_constant__ Inst I, const float *__restrict__ f0,
                             float *__restrict__ lam) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const uint32_t pk = S.node[t];
  if (pk == kNoNode) return;
  int x, y, z;
  unpack(pk, x, y, z);
  if (z != I.L.nz - 1) return;
  const unsigned ns = (unsigned)S.ns;
  const unsigned gs = (unsigned)(I.ghost + I.L.plane) + (unsigned)(y * I.L.nx + x);
  float fr[Q], fp[Q], gr[Q], gp[Q], lr[Q], lp[Q];
  for (int i = 0; i < Q; ++i) {
    Store<float>::ld2(f0, ns, i, t, i, fr[i], fp[i]);   // the start state, in the slot layout
    gr[i] = CZ[i] == -1 ? lam[(unsigned)i * ns + gs] : 0.f;
    gp[i] = CZ[i] == -1 ? lam[(unsigned)(Q + i) * ns + gs] : 0.f;
    lr[i] = lam[(unsigned)i * ns + t];
    lp[i] = lam[(unsigned)(Q + i) * ns + t];
  }
  outlet_ghost_adj(fr, fp, I.P.rho_out, gr, gp, lr, lp);
  for (int i = 0; i < Q; ++i) {
    lam[(unsigned)i * ns + t] = lr[i];
    lam[(unsigned)(Q + i) * ns + t] = lp[i];
  }
  lam[(unsigned)(2 * Q + 5) * ns + t] += lam[(unsigned)(2 * Q + 5) * ns + gs];
}

}  // namespace cglbm
