// Device functions of the freeform-lens trace: counter-based ray generation,
// B-spline patch evaluation, refraction, propagation, the reconstruction filter
// and the reverse-mode derivatives of all of them.
#pragma once

#include <cstdint>

#include "fr_internal.h"

namespace fr {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (id_lo, id_hi,
// 0, 0), key = seed. Ten rounds of two 32x32->64-bit products; the key is bumped
// by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint2 philox_ray_words(uint64_t seed, uint64_t id) {
  uint32_t c0 = (uint32_t)id, c1 = (uint32_t)(id >> 32), c2 = 0u, c3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint2(c0, c1);
}

// Top 23 bits of a word plus one half, times 2^-23: exact in FP32, in (0,1).
__device__ __forceinline__ float unit23(uint32_t w) {
  return fmaf((float)(w >> 9), 1.0f / 8388608.0f, 0.5f / 8388608.0f);
}

// ---------------------------------------------------------------------------
// Sec. 2.1: the bicubic B-spline height field as power-form patches. On span
// product (k, l) with local coordinates s, t in [0,1],
//   Z(s,t) = sum_{e,f} C[e][f] s^e t^f,
// where C is the prep kernel's exact re-expression of sum N_i N_j P^z_ij.
// ---------------------------------------------------------------------------
struct Patch {
  int k, l;
  float4 c0, c1, c2, c3;   // c_e = (C[e][0], C[e][1], C[e][2], C[e][3])
};

__device__ __forceinline__ void locate(float u, int ns, int* k, float* s) {
  const float us = fminf(fmaxf(u, 0.0f), 1.0f) * (float)ns;
  const int kk = min((int)us, ns - 1);
  *k = kk;
  *s = us - (float)kk;
}

__device__ __forceinline__ void fetch_patch(const float4* sp, int nsv, int k, int l, Patch* p) {
  if (k != p->k || l != p->l) {
    const float4* q = sp + (size_t)(k * nsv + l) * 4;
    p->c0 = q[0];
    p->c1 = q[1];
    p->c2 = q[2];
    p->c3 = q[3];
    p->k = k;
    p->l = l;
  }
}

// One cubic in t and its derivative (Horner with synthetic division).
__device__ __forceinline__ void cubic_d(const float4 c, float t, float* v, float* dv) {
  const float a = fmaf(t, c.w, c.z);
  const float b = fmaf(t, a, c.y);
  const float db = fmaf(t, c.w, a);
  *v = fmaf(t, b, c.x);
  *dv = fmaf(t, db, b);
}

// Z, dZ/ds, dZ/dt.
__device__ __forceinline__ void patch_eval(const Patch& p, float s, float t, float* Z, float* Zs, float* Zt) {
  float r0, r1, r2, r3, d0, d1, d2, d3;
  cubic_d(p.c0, t, &r0, &d0);
  cubic_d(p.c1, t, &r1, &d1);
  cubic_d(p.c2, t, &r2, &d2);
  cubic_d(p.c3, t, &r3, &d3);
  const float a = fmaf(s, r3, r2);
  const float b = fmaf(s, a, r1);
  const float db = fmaf(s, r3, a);
  *Z = fmaf(s, b, r0);
  *Zs = fmaf(s, db, b);
  *Zt = fmaf(s, fmaf(s, fmaf(s, d3, d2), d1), d0);
}

// Second derivatives d2Z/ds2, d2Z/dsdt, d2Z/dt2.
__device__ __forceinline__ void patch_eval2(const Patch& p, float s, float t, float* Zss, float* Zst, float* Ztt) {
  float r2, r3, d1, d2, d3, tmp;
  cubic_d(p.c1, t, &tmp, &d1);
  cubic_d(p.c2, t, &r2, &d2);
  cubic_d(p.c3, t, &r3, &d3);
  *Zss = fmaf(6.0f * s, r3, 2.0f * r2);
  *Zst = fmaf(s, fmaf(3.0f * s, d3, 2.0f * d2), d1);
  // d2/dt2 of each row cubic: 2 c_e2 + 6 c_e3 t
  const float e0 = fmaf(6.0f * t, p.c0.w, 2.0f * p.c0.z);
  const float e1 = fmaf(6.0f * t, p.c1.w, 2.0f * p.c1.z);
  const float e2 = fmaf(6.0f * t, p.c2.w, 2.0f * p.c2.z);
  const float e3 = fmaf(6.0f * t, p.c3.w, 2.0f * p.c3.z);
  *Ztt = fmaf(s, fmaf(s, fmaf(s, e3, e2), e1), e0);
}

// The four non-zero basis functions N_{k+a}(s) of a span and dN/ds from the
// prep kernel's power-form table.
__device__ __forceinline__ void basis_eval(const float4* tab, float s, float N[4], float dN[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) cubic_d(tab[a], s, &N[a], &dN[a]);
}

// ---------------------------------------------------------------------------
// One ray up to the screen (Secs. 2.2-2.3). Everything the adjoint needs is
// kept, so that forward and adjoint run the same code.
// ---------------------------------------------------------------------------
struct RayFwd {
  int status;
  int iters;
  float u, v;           // hit in the B-spline parameter domain
  float s, t;           // patch coordinates of the hit (patch in the Patch cache)
  float x, y, z;        // hit on the freeform
  float dx, dy, dz;     // direction inside the glass
  float Zs, Zt;         // surface derivatives in patch coordinates at the hit
  float nx, ny, nz;     // unit normal (into the air)
  float invL;           // 1/|(-Z_x,-Z_y,1)|
  float c, cs, a;       // cos(incidence) d.n, cos(transmission), eta c - cs
  float tx, ty, tz;     // direction after the freeform
  float T1, T2, w;      // Schlick transmissions and final weight
  float lam;            // distance parameter to the screen
  float X, Y;           // screen hit
  float tstar, gp;      // point source: ray parameter of the hit and df/dt there
};

// Exit face: normal, Snell glass -> air, TIR, Schlick, propagation (a5, a6).
__device__ __forceinline__ void exit_and_propagate(const Item& it, RayFwd& r) {
  const float Zx = r.Zs * it.ku, Zy = r.Zt * it.kv;
  const float invL = rsqrtf(fmaf(Zx, Zx, fmaf(Zy, Zy, 1.0f)));
  r.invL = invL;
  r.nx = -Zx * invL;
  r.ny = -Zy * invL;
  r.nz = invL;
  const float eta = it.n_glass;
  const float c = fmaf(r.dx, r.nx, fmaf(r.dy, r.ny, r.dz * r.nz));
  r.c = c;
  const float k = fmaf(-eta * eta, fmaf(-c, c, 1.0f), 1.0f);
  if (!(k >= 0.0f)) { r.status = FR_RAY_TIR; return; }
  const float cs = sqrtf(k);
  r.cs = cs;
  const float a = fmaf(eta, c, -cs);
  r.a = a;
  r.tx = fmaf(eta, r.dx, -a * r.nx);
  r.ty = fmaf(eta, r.dy, -a * r.ny);
  r.tz = fmaf(eta, r.dz, -a * r.nz);
  const float om = 1.0f - cs;
  const float om2 = om * om;
  r.T2 = (1.0f - it.R0) * fmaf(-om2 * om2, om, 1.0f);
  r.w = it.omega0 * r.T1 * r.T2;
  if (!(r.tz > 0.0f)) { r.status = FR_RAY_OFF_SCREEN; return; }
  const float lam = __fdividef(it.z_screen - r.z, r.tz);
  r.lam = lam;
  r.X = fmaf(lam, r.tx, r.x);
  r.Y = fmaf(lam, r.ty, r.y);
  if (!(fabsf(r.X) < it.Rx && fabsf(r.Y) < it.Ry)) { r.status = FR_RAY_OFF_SCREEN; return; }
  r.status = FR_RAY_ON_SCREEN;
}

// Collimated ray (a1, a3-a6): (u,v) on the square grid, d = (0,0,1), starting
// on the freeform.
__device__ __forceinline__ void trace_collimated(const Item& it, const float4* sp, Patch& pc, int row, int col,
                                                 uint64_t id, float inv_cols, float inv_rows, RayFwd& r) {
  float ja = 0.5f, jb = 0.5f;
  if (it.jitter) {
    const uint2 w = philox_ray_words(it.seed, id);
    ja = unit23(w.x);
    jb = unit23(w.y);
  }
  const float u = ((float)col + ja) * inv_cols;
  const float v = ((float)row + jb) * inv_rows;
  r.u = u;
  r.v = v;
  r.x = fmaf(2.0f, u, -1.0f) * it.rx;
  r.y = fmaf(2.0f, v, -1.0f) * it.ry;
  int k, l;
  locate(u, it.nsu, &k, &r.s);
  locate(v, it.nsv, &l, &r.t);
  fetch_patch(sp, it.nsv, k, l, &pc);
  float Z;
  patch_eval(pc, r.s, r.t, &Z, &r.Zs, &r.Zt);
  r.z = Z;
  r.dx = 0.0f;
  r.dy = 0.0f;
  r.dz = 1.0f;
  r.T1 = 1.0f - it.R0;   // normal incidence on the flat entry face
  r.iters = 0;
  exit_and_propagate(it, r);
}

// f(t) = Z(o_uv + d_uv t) - o_z - d_z t (Eq. surfaceintersect) and df/dt.
__device__ __forceinline__ void f_eval(const Item& it, const float4* sp, Patch& pc, float ou, float ov, float du,
                                       float dv, float oz, float dz, float t, RayFwd& r, float* f, float* fp) {
  int k, l;
  locate(fmaf(du, t, ou), it.nsu, &k, &r.s);
  locate(fmaf(dv, t, ov), it.nsv, &l, &r.t);
  fetch_patch(sp, it.nsv, k, l, &pc);
  float Z;
  patch_eval(pc, r.s, r.t, &Z, &r.Zs, &r.Zt);
  *f = Z - fmaf(dz, t, oz);
  *fp = fmaf(r.Zs, du * (float)it.nsu, fmaf(r.Zt, dv * (float)it.nsv, -dz));
}

// Point source (a1, a2, a4-a6): Philox direction uniform in the cone, flat
// entry face, Snell + Schlick into the glass, safeguarded Newton on f(t)
// bracketed by the convex hull of the control heights (Sec. 2.1.2).
__device__ __forceinline__ void trace_point(const Item& it, const float4* sp, Patch& pc, uint64_t id, float zmin,
                                            float zmax, RayFwd& r) {
  r.iters = 0;
  const uint2 w = philox_ray_words(it.seed, id);
  const float xi1 = unit23(w.x), xi2 = unit23(w.y);
  float sx = it.px, sy = it.py;
  if (it.gnx * it.gny > 1) {
    uint32_t src = (uint32_t)(id / it.per_src);
    src = min(src, (uint32_t)(it.gnx * it.gny - 1));
    const uint32_t gx = src % (uint32_t)it.gnx, gy = src / (uint32_t)it.gnx;
    sx += fmaf((float)gx, it.gdx, it.gx0);
    sy += fmaf((float)gy, it.gdy, it.gy0);
  }
  float sn, cn;
  sincospif(2.0f * xi1, &sn, &cn);
  const float omc = it.omc_max * xi2;            // 1 - cos(phi)
  const float sphi = sqrtf(omc * (2.0f - omc));
  const float d0x = cn * sphi, d0y = sn * sphi, d0z = 1.0f - omc;
  const float tau = __fdividef(it.z_in - it.pz, d0z);
  const float ox = fmaf(tau, d0x, sx), oy = fmaf(tau, d0y, sy), oz = it.z_in;
  if (!(tau > 0.0f) || fabsf(ox) > it.rx || fabsf(oy) > it.ry) { r.status = FR_RAY_APERTURE_MISS; return; }
  // Snell air -> glass at the flat face, normal (0,0,1).
  const float eta1 = 1.0f / it.n_glass;
  r.dx = eta1 * d0x;
  r.dy = eta1 * d0y;
  r.dz = sqrtf(fmaf(-eta1 * eta1, sphi * sphi, 1.0f));
  const float om2 = omc * omc;
  r.T1 = (1.0f - it.R0) * fmaf(-om2 * om2, omc, 1.0f);
  // Bracket: the slab zmin <= z <= zmax, widened a little for FP32 rounding,
  // cut where the ray leaves the domain [0,1]^2 (the side of the lens).
  const float pad = 1e-6f * (1.0f + fmaxf(fabsf(zmin), fabsf(zmax)));
  const float inv_dz = 1.0f / r.dz;
  float ta = fmaxf(0.0f, (zmin - pad - oz) * inv_dz);
  const float t_hi = (zmax + pad - oz) * inv_dz;
  const float ou = fmaf(0.5f / it.rx, ox, 0.5f), ov = fmaf(0.5f / it.ry, oy, 0.5f);
  const float du = r.dx * (0.5f / it.rx), dv = r.dy * (0.5f / it.ry);
  float t_dom = INFINITY;
  if (du > 0.0f) t_dom = fminf(t_dom, (1.0f - ou) / du);
  if (du < 0.0f) t_dom = fminf(t_dom, -ou / du);
  if (dv > 0.0f) t_dom = fminf(t_dom, (1.0f - ov) / dv);
  if (dv < 0.0f) t_dom = fminf(t_dom, -ov / dv);
  if (t_dom < ta) { r.status = FR_RAY_OUT_OF_DOMAIN; return; }
  float tb = fminf(t_hi, t_dom);
  float f, fp;
  if (tb < t_hi) {
    f_eval(it, sp, pc, ou, ov, du, dv, oz, r.dz, tb, r, &f, &fp);
    if (f > 0.0f) { r.status = FR_RAY_OUT_OF_DOMAIN; return; }   // leaves the side first
  }
  float t = ta;
  f_eval(it, sp, pc, ou, ov, du, dv, oz, r.dz, t, r, &f, &fp);
  if (f < 0.0f) { r.status = FR_RAY_INVALID; return; }
  bool converged = (f == 0.0f);
  for (int it_n = 0; it_n < it.newton_max && !converged; ++it_n) {
    float tn = t - __fdividef(f, fp);
    if (!(fp < 0.0f) || !(tn > ta && tn < tb)) tn = 0.5f * (ta + tb);
    const float step = fabsf(tn - t);
    t = tn;
    f_eval(it, sp, pc, ou, ov, du, dv, oz, r.dz, t, r, &f, &fp);
    r.iters = it_n + 1;
    if (f > 0.0f) ta = t; else tb = t;
    if (step <= it.newton_tol || f == 0.0f) converged = true;
  }
  if (!converged) { r.status = FR_RAY_NEWTON_FAIL; return; }
  r.tstar = t;
  r.gp = fp;
  r.u = fmaf(du, t, ou);
  r.v = fmaf(dv, t, ov);
  r.x = fmaf(r.dx, t, ox);
  r.y = fmaf(r.dy, t, oy);
  r.z = fmaf(r.dz, t, oz);
  exit_and_propagate(it, r);
}

// ---------------------------------------------------------------------------
// Sec. 2.3: Gaussian reconstruction filter on the nu x nu footprint around the
// pixel that holds the hit; every other pixel has f = 0.
// ---------------------------------------------------------------------------
template <int NU>
struct Foot {
  int ie, je;           // extended column / row of the footprint's first cell
  float gx, gy;         // hit in extended pixel units
  float fx[NU], fy[NU]; // filter values
  float rsx, rsy;       // 1 / sum f
};

template <int NU>
__device__ __forceinline__ bool footprint(const Item& it, float X, float Y, Foot<NU>& f) {
  constexpr int h = (NU - 1) / 2;
  const float gx = (X + it.Rsx) * it.inv_wx;
  const float gy = (Y + it.Rsy) * it.inv_wy;
  const int ic = min(max((int)floorf(gx), h), it.nx + h - 1);
  const int jc = min(max((int)floorf(gy), h), it.ny + h - 1);
  f.gx = gx;
  f.gy = gy;
  f.ie = ic - h;
  f.je = jc - h;
  float sx = 0.0f, sy = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    const float dxa = gx - ((float)(f.ie + a) + 0.5f);
    const float dya = gy - ((float)(f.je + a) + 0.5f);
    f.fx[a] = fabsf(dxa) < 0.5f * NU ? exp2f(-it.ax * dxa * dxa) - it.cut : 0.0f;
    f.fy[a] = fabsf(dya) < 0.5f * NU ? exp2f(-it.ay * dya * dya) - it.cut : 0.0f;
    sx += f.fx[a];
    sy += f.fy[a];
  }
  if (!(sx > 0.0f) || !(sy > 0.0f)) return false;  // nu = 1 exactly on a pixel edge
  f.rsx = 1.0f / sx;
  f.rsy = 1.0f / sy;
  return true;
}

// ---------------------------------------------------------------------------
// Reverse mode of one ray (a9). Input: G[b][a] = dL/dE on the footprint (row b,
// column a). Output: the adjoint zeta of the hit height and of the surface
// slopes, from which dL/dP^z_{k+a,l+b} = zeta N_a N_b + Zs_bar N'_a N_b
// + Zt_bar N_a N'_b.
// ---------------------------------------------------------------------------
template <int NU>
__device__ __forceinline__ void ray_reverse(const Item& it, const RayFwd& r, const Foot<NU>& f,
                                            const float (&G)[NU][NU], bool point, const Patch& pc,
                                            float* zeta, float* Zs_bar, float* Zt_bar) {
  // Filter: F_a = f_a / S, dF_a/dX = (f'_a - F_a S') / S with f'_a = -2 alpha delta_a e_a / w.
  const float ln2 = 0.69314718055994531f;
  float Fx[NU], Fy[NU], gxa[NU], gya[NU];
  float Spx = 0.0f, Spy = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    const float dxa = f.gx - ((float)(f.ie + a) + 0.5f);
    const float dya = f.gy - ((float)(f.je + a) + 0.5f);
    // exp part e = f + cut inside the support, its derivative in world units
    gxa[a] = f.fx[a] != 0.0f ? -2.0f * (it.ax * ln2) * dxa * (f.fx[a] + it.cut) * it.inv_wx : 0.0f;
    gya[a] = f.fy[a] != 0.0f ? -2.0f * (it.ay * ln2) * dya * (f.fy[a] + it.cut) * it.inv_wy : 0.0f;
    Spx += gxa[a];
    Spy += gya[a];
    Fx[a] = f.fx[a] * f.rsx;
    Fy[a] = f.fy[a] * f.rsy;
  }
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    // With nu = 1 the normalised filter is identically 1 on its pixel: its
    // derivative is exactly 0 (the general formula leaves rounding noise).
    gxa[a] = NU == 1 ? 0.0f : (gxa[a] - Fx[a] * Spx) * f.rsx;
    gya[a] = NU == 1 ? 0.0f : (gya[a] - Fy[a] * Spy) * f.rsy;
  }
  float wbar = 0.0f, Xs = 0.0f, Ys = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int b = 0; b < NU; ++b) {
      A = fmaf(G[b][a], Fy[b], A);
      B = fmaf(G[b][a], gya[b], B);
    }
    wbar = fmaf(A, Fx[a], wbar);
    Xs = fmaf(A, gxa[a], Xs);
    Ys = fmaf(B, Fx[a], Ys);
  }
  const float K = r.w * it.inv_area;
  wbar *= it.inv_area;
  const float Xbar = K * Xs, Ybar = K * Ys;
  // Propagation X = x + lam t_x, lam = (z_s - z)/t_z.
  float txb = r.lam * Xbar, tyb = r.lam * Ybar;
  const float lamb = fmaf(Xbar, r.tx, Ybar * r.ty);
  const float inv_tz = 1.0f / r.tz;
  float tzb = -lamb * r.lam * inv_tz;
  const float zbar = -lamb * inv_tz;
  // Weight w = omega0 T1 T2, T2 = (1-R0)(1-(1-cs)^5).
  const float om = 1.0f - r.cs;
  const float om2 = om * om;
  float csb = wbar * it.omega0 * r.T1 * (1.0f - it.R0) * 5.0f * om2 * om2;
  // Refraction t = eta d - a n, a = eta c - cs, cs = sqrt(1 - eta^2 (1 - c^2)), c = d.n.
  const float eta = it.n_glass;
  const float abar = -(txb * r.nx + tyb * r.ny + tzb * r.nz);
  float nbx = -r.a * txb, nby = -r.a * tyb, nbz = -r.a * tzb;
  float cbar = eta * abar;
  csb -= abar;
  const float kbar = csb * 0.5f / r.cs;
  cbar = fmaf(kbar * 2.0f * eta * eta, r.c, cbar);
  nbx = fmaf(cbar, r.dx, nbx);
  nby = fmaf(cbar, r.dy, nby);
  nbz = fmaf(cbar, r.dz, nbz);
  // Normalisation n = m / |m|, m = (-Z_x, -Z_y, 1).
  const float ndot = nbx * r.nx + nby * r.ny + nbz * r.nz;
  const float mbx = (nbx - ndot * r.nx) * r.invL;
  const float mby = (nby - ndot * r.ny) * r.invL;
  *Zs_bar = -mbx * it.ku;
  *Zt_bar = -mby * it.kv;
  if (!point) {
    *zeta = zbar;   // the hit height is Z itself
    return;
  }
  // Point source: the hit moves along the ray with t*; implicit function
  // theorem on f(t*, P) = 0 gives dt*/dP_ab = -N_a N_b / f'(t*).
  float Zss, Zst, Ztt;
  patch_eval2(pc, r.s, r.t, &Zss, &Zst, &Ztt);
  const float dsdt = r.dx * (0.5f / it.rx) * (float)it.nsu;
  const float dtdt = r.dy * (0.5f / it.ry) * (float)it.nsv;
  const float tbar = Xbar * r.dx + Ybar * r.dy + zbar * r.dz +
                     *Zs_bar * fmaf(Zss, dsdt, Zst * dtdt) + *Zt_bar * fmaf(Zst, dsdt, Ztt * dtdt);
  *zeta = -tbar / r.gp;
}

// Per-thread ray counts by cause (FR_RAY_*), summed per CTA and added to the
// caller's fr_stats once per CTA.
struct Counters {
  unsigned int n[FR_RAY_NCAUSES];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int s = 0; s < FR_RAY_NCAUSES; ++s) n[s] = 0u;
  }
  __device__ __forceinline__ void add(int status) {
#pragma unroll
    for (int s = 0; s < FR_RAY_NCAUSES; ++s) n[s] += (status == s) ? 1u : 0u;
  }
  // Warp sums, then one shared atomic per warp and cause (all lanes active).
  __device__ __forceinline__ void reduce_into(unsigned int* s_cnt) const {
#pragma unroll
    for (int s = 0; s < FR_RAY_NCAUSES; ++s) {
      const unsigned int v = __reduce_add_sync(0xffffffffu, n[s]);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[s], v);
    }
  }
  // After a __syncthreads that follows reduce_into.
  static __device__ __forceinline__ void publish(const unsigned int* s_cnt, fr_stats* stats) {
    if (stats && threadIdx.x < FR_RAY_NCAUSES && s_cnt[threadIdx.x])
      atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rays[threadIdx.x]),
                (unsigned long long)s_cnt[threadIdx.x]);
  }
};

}  // namespace fr
