// Persistent velocity-block sweep of one UGKS time step.
//
// One persistent CTA per SM owns a few spatial tiles of cells (contiguous in
// the locality order built at create time) and sweeps every velocity block m
// of BV = 32 points (Sec. 2.2.2, Eq. 48; one warp lane per velocity), tile by
// tile, so that all CTAs advance through the blocks together and a tile's
// halo rows are still in L2 when its neighbours read them:
//   phase G  limited least-squares gradients of h, b for the tile cells and
//            their face neighbours (reconstruction, Eq. 31)        [Table B.1 K2]
//   phase F  time-integrated micro fluxes of every face touching the tile
//            (Eq. 29, 33-35), warp-shuffle reduction of their weighted
//            moments into per-face FP64 accumulators (Eq. 52, Algorithm 4)
//   phase S  first-stage update of the tile cells (Eq. 41, Algorithm 1)
// then, without leaving the kernel, the conservative update (Eq. 27) of its
// own cells from the face accumulators and the second-stage update (Eq. 42)
// of their distributions, which also accumulates the heat flux of f^{n+1}
// (Eq. 13) for the next step.
//
// Faces shared by two tiles are evaluated by both with the same instruction
// sequence, so both tiles see the same flux and W stays exactly conservative;
// no CTA waits on another.  f^n is read-only during the step (f~ and f^{n+1}
// go to the second buffer), so neighbour reads need no synchronisation.  The
// gradients and micro fluxes of the current tile and block live in shared
// memory (the tile size is chosen so that they fit); only the FP64 face
// accumulators of the CTA's tiles live in global memory (they stay in L2).
#include <cmath>
#include <cstdint>
#include <mutex>

#include "ugks_device.cuh"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"

namespace ugks {

template <int D, int NR, typename T>
__global__ void __launch_bounds__(1024, 1) k_sweep(SweepArgs<T> a) {
  constexpr int NW = D + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const sG = reinterpret_cast<T*>(smem_raw);        // [gset][NR][D][BV] of the current tile
  T* const sPhi = sG + a.smem_g_elems;                  // [faces][NR][BV] of the current tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t Nc = a.Nc, M = a.M;
  const T dt = T(a.g.dt);
  const T hdt2 = T(0.5 * a.g.dt * a.g.dt);
  const int limiter = a.g.limiter;
  const int Kxi = a.g.Kxi;
  const int idx8 = sum8_index(lane);
  const bool writer8 = (lane & 3) == 0;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    double* Facc = a.Facc + size_t(tile) * a.Facc_stride;
    const int nfc = int(a.tf_off[tile + 1] - a.tf_off[tile]);
    for (int i = threadIdx.x; i < nfc * FACC_W; i += blockDim.x) Facc[i] = 0.0;
  }
  __syncthreads();

  for (int64_t m = 0; m < M; ++m) {
    const int64_t k = m * BV + lane;
    T u[3];
    u[0] = a.ux[k];
    u[1] = D > 1 ? a.uy[k] : T(0);
    u[2] = D > 2 ? a.uz[k] : T(0);
    const T wk = a.w[k];
    const bool real_v = k < a.nv;
    const T wi = real_v ? wk : T(0);
    T u2 = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) u2 += u[d] * u[d];

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      const int64_t c0 = a.tile_begin[tile], c1 = a.tile_begin[tile + 1];
      const int nt = int(c1 - c0);
      const int64_t* gset = a.gset + a.gset_off[tile];
      const int ng = int(a.gset_off[tile + 1] - a.gset_off[tile]);
      const TileFace* tf = a.tf + a.tf_off[tile];
      const int nfc = int(a.tf_off[tile + 1] - a.tf_off[tile]);
      double* Facc = a.Facc + size_t(tile) * a.Facc_stride;

      // ---- phase G: limited least-squares gradients (reconstruction, Eq. 31) ----
      for (int li = warp; li < ng; li += nwarps) {
        const int64_t c = gset[li];
        T fc[NR], g[NR][D], fmx[NR], fmn[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          fc[r] = a.f_cur[frow(r, m, c, M, Nc) + lane];
          fmx[r] = fmn[r] = fc[r];
#pragma unroll
          for (int d = 0; d < D; ++d) g[r][d] = T(0);
        }
        const int64_t e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
        for (int64_t e = e0; e < e1; ++e) {
          const CellFaceT<T> s = a.cf[e];
          if (s.flags & 1) continue;  // walls: one-sided
          T fo[NR];
          if (s.other >= 0) {
#pragma unroll
            for (int r = 0; r < NR; ++r) fo[r] = a.f_cur[frow(r, m, s.other, M, Nc) + lane];
          } else {
            const BCDev& bc = a.bcs[s.bc];
            T rho, lam, U[3];
            if (bc.type == 3) {
              const CellPrim& p = a.cp[c];
              rho = T(p.rho); lam = T(p.lam);
              U[0] = T(p.U[0]); U[1] = T(p.U[1]); U[2] = T(p.U[2]);
            } else {
              rho = T(bc.rho); lam = T(1.0 / bc.T);
              U[0] = T(bc.u[0]); U[1] = T(bc.u[1]); U[2] = T(bc.u[2]);
            }
            T c2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) c2 += (u[d] - U[d]) * (u[d] - U[d]);
            const T H = real_v ? rho * maxwell_pref<D>(lam) * t_exp(-lam * c2) : T(0);
            fo[0] = H;
            if (NR == 2) fo[NR - 1] = T(Kxi) / (T(2) * lam) * H;
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const T df = fo[r] - fc[r];
#pragma unroll
            for (int d = 0; d < D; ++d) g[r][d] += s.w[d] * df;
            fmx[r] = fmax(fmx[r], fo[r]);
            fmn[r] = fmin(fmn[r], fo[r]);
          }
        }
        T phi[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) phi[r] = T(1);
        if (limiter != 0) {
          const T eps2c = a.eps2[c];
          T eps2[NR], dmx[NR], dmn[NR];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const T mag = fmax(fabs(fmx[r]), fabs(fmn[r]));
            eps2[r] = eps2c * mag * mag;  // Venkatakrishnan constant in the units of f
            dmx[r] = fmx[r] - fc[r];
            dmn[r] = fmn[r] - fc[r];
          }
          for (int64_t e = e0; e < e1; ++e) {
            const CellFaceT<T> s = a.cf[e];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              T d2 = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) d2 += g[r][d] * s.r[d];
              const T dp = d2 > T(0) ? dmx[r] : dmn[r];
              T ph;
              if (limiter == 2) {
                ph = d2 != T(0) ? fast_div(dp, d2) : T(1);
              } else {
                // (dp^2 + eps + 2 d2 dp) / (dp^2 + 2 d2^2 + dp d2 + eps); equals 1 at d2 = 0
                const T num = fma(dp, dp + T(2) * d2, eps2[r]);
                const T den = fma(dp + d2, dp, fma(T(2) * d2, d2, eps2[r]));
                ph = fast_div(num, den);
              }
              phi[r] = fmin(phi[r], ph);  // fmin ignores a NaN from 0/0 (then d2 = 0, phi stays)
            }
          }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const T p = fmin(fmax(phi[r], T(0)), T(1));
#pragma unroll
          for (int d = 0; d < D; ++d) sG[((size_t(li) * NR + r) * D + d) * BV + lane] = p * g[r][d];
        }
      }
      __syncthreads();

      // ---- phase F: micro fluxes and their moments (Eq. 29, 33-35, 52; Algorithm 4) ----
      for (int lf = warp; lf < nfc; lf += nwarps) {
        const TileFace t = tf[lf];
        double* Fa = Facc + size_t(lf) * FACC_W;
        const double fold = (writer8 && idx8 < NW) ? Fa[idx8] : 0.0;  // issued early, used at the end
        const FaceGeom<T> fg = a.fg[t.face];
        const FaceRec<T> R = a.fr[t.face];
        T un = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) un += u[d] * fg.n[d];
        T phi_h = T(0), phi_b = T(0);
        if (fg.bc_type == 1) {
          // diffuse wall (Eq. 36-38; free transport f(x - u t) on the incoming side)
          const double fold_out = (writer8 && idx8 < NW) ? Fa[5 + idx8] : 0.0;
          T out_h = T(0);
          if (un > T(0)) {
            T v[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              T fin = a.f_cur[frow(r, m, fg.own, M, Nc) + lane], ug = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) {
                const T gd = sG[((size_t(t.lo) * NR + r) * D + d) * BV + lane];
                fin += gd * fg.rl[d];
                ug += u[d] * gd;
              }
              v[r] = dt * fin - hdt2 * ug;
            }
            phi_h = un * v[0];
            if (NR == 2) phi_b = un * v[NR - 1];
          } else if (un < T(0)) {
            T c2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) c2 += (u[d] - R.U[d]) * (u[d] - R.U[d]);
            out_h = un * dt * R.rho_pref * t_exp(-R.lam * c2);
          }
          const T wph = wi * phi_h, wpo = wi * out_h;
          const T sin = warp_sum8<T>(wph, wph * u[0], D > 1 ? wph * u[1] : energy_in(D, wi, u2, phi_h, phi_b),
                                     D > 2 ? wph * u[2] : (D == 2 ? energy_in(D, wi, u2, phi_h, phi_b) : T(0)),
                                     D > 2 ? energy_in(D, wi, u2, phi_h, phi_b) : T(0), T(0), T(0), T(0), lane);
          const T eo = T(0.5) * wi * (u2 * out_h + R.kappa * out_h);
          const T sout = warp_sum8<T>(wpo, wpo * u[0], D > 1 ? wpo * u[1] : eo, D > 2 ? wpo * u[2] : (D == 2 ? eo : T(0)),
                                      D > 2 ? eo : T(0), T(0), T(0), T(0), lane);
          if (writer8 && idx8 < NW) {
            Fa[idx8] = fold + double(sin);
            Fa[5 + idx8] = fold_out + double(sout);
          }
        } else {
          if (un != T(0)) {
            T fs[NR], gs[NR][D], off[D];
            const bool left = un > T(0);
            if (left || t.ln >= 0) {
              const int64_t cs = left ? fg.own : fg.nei;
              const int ls = left ? t.lo : t.ln;
#pragma unroll
              for (int d = 0; d < D; ++d) off[d] = left ? fg.rl[d] : fg.rr[d];
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                fs[r] = a.f_cur[frow(r, m, cs, M, Nc) + lane];
#pragma unroll
                for (int d = 0; d < D; ++d) gs[r][d] = sG[((size_t(ls) * NR + r) * D + d) * BV + lane];
              }
            } else {
              // ghost side of an artificial boundary: Maxwellian of the ghost state, no slope
              const BCDev& bc = a.bcs[-fg.nei - 1];
              T rho, lam, U[3];
              if (bc.type == 3) {
                const CellPrim& p = a.cp[fg.own];
                rho = T(p.rho); lam = T(p.lam);
                U[0] = T(p.U[0]); U[1] = T(p.U[1]); U[2] = T(p.U[2]);
              } else {
                rho = T(bc.rho); lam = T(1.0 / bc.T);
                U[0] = T(bc.u[0]); U[1] = T(bc.u[1]); U[2] = T(bc.u[2]);
              }
              T c2 = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) c2 += (u[d] - U[d]) * (u[d] - U[d]);
              const T H = rho * maxwell_pref<D>(lam) * t_exp(-lam * c2);
              fs[0] = H;
              if (NR == 2) fs[NR - 1] = T(Kxi) / (T(2) * lam) * H;
#pragma unroll
              for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int d = 0; d < D; ++d) gs[r][d] = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) off[d] = T(0);
            }
            // free-transport part: G0 f_face + G1 u.grad f (Eq. 31, 33)
            T tr[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              T ff = fs[r], ug = T(0);
#pragma unroll
              for (int d = 0; d < D; ++d) {
                ff += gs[r][d] * off[d];
                ug += u[d] * gs[r][d];
              }
              tr[r] = R.G[0] * ff + R.G[1] * ug;
            }
            // equilibrium part: G2 (g0 + g0+) + G3 u.grad g0 + G4 d_t g0 (Eq. 32-33)
            T cc[3], c2 = T(0), cq = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              cc[d] = u[d] - R.U[d];
              c2 += cc[d] * cc[d];
              cq += cc[d] * R.q[d];
            }
            const T H0 = R.rho_pref * t_exp(-R.lam * c2);
            const T sq = R.sq * cq;
            const T twolc2 = T(2) * R.lam * c2;
            const T h0 = H0 * (T(1) + sq * (twolc2 - T(2 + D)));
            T ugH = T(0), ugB = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              T poly = R.a[d][0] + T(0.5) * R.a[d][D + 1] * u2;
#pragma unroll
              for (int e = 0; e < D; ++e) poly += R.a[d][1 + e] * u[e];
              ugH += u[d] * (poly + T(0.5) * R.a[d][D + 1] * R.kappa);
              if (NR == 2) ugB += u[d] * (poly * R.kappa + T(0.5) * R.a[d][D + 1] * R.xi4);
            }
            T pA = R.A[0] + T(0.5) * R.A[D + 1] * u2;
#pragma unroll
            for (int e = 0; e < D; ++e) pA += R.A[1 + e] * u[e];
            const T dtH = pA + T(0.5) * R.A[D + 1] * R.kappa;
            phi_h = un * (tr[0] + R.G[2] * h0 + H0 * (R.G[3] * ugH + R.G[4] * dtH));
            if (NR == 2) {
              const T b0 = H0 * R.kappa * (T(1) + sq * (twolc2 - T(D)));
              const T dtB = pA * R.kappa + T(0.5) * R.A[D + 1] * R.xi4;
              phi_b = un * (tr[NR - 1] + R.G[2] * b0 + H0 * (R.G[3] * ugB + R.G[4] * dtB));
            }
          }
          const T wph = wi * phi_h;
          const T en = T(0.5) * wi * (u2 * phi_h + phi_b);
          // value index t of the reduction is conservative variable t (energy at D + 1)
          const T sm = warp_sum8<T>(wph, wph * u[0], D > 1 ? wph * u[1] : en, D > 2 ? wph * u[2] : (D == 2 ? en : T(0)),
                                    D > 2 ? en : T(0), T(0), T(0), T(0), lane);
          if (writer8 && idx8 < NW) Fa[idx8] = fold + double(sm);
        }
        sPhi[(size_t(lf) * NR + 0) * BV + lane] = phi_h;
        if (NR == 2) sPhi[(size_t(lf) * NR + NR - 1) * BV + lane] = phi_b;
      }
      __syncthreads();

      // ---- phase S: first-stage update of the tile cells (Eq. 41; Algorithm 1) ----
      for (int li = warp; li < nt; li += nwarps) {
        const int64_t c = c0 + li;
        const CellPrim& p = a.cp[c];
        const T rho = T(p.rho), lam = T(p.lam), beta0 = dt / (T(2) * T(p.tau));
        T c2 = T(0), cq = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const T cd = u[d] - T(p.U[d]);
          c2 += cd * cd;
          cq += cd * T(p.q[d]);
        }
        const T H = rho * maxwell_pref<D>(lam) * t_exp(-lam * c2);
        const T s = a.g.shakhov ? T(4.0 * (1.0 - a.g.Pr)) * lam * lam / (T(5) * rho) * cq : T(0);
        T fp[NR];
        fp[0] = H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)));
        if (NR == 2) fp[NR - 1] = T(Kxi) / (T(2) * lam) * H * (T(1) + s * (T(2) * lam * c2 - T(D)));
        T flux[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) flux[r] = T(0);
        const int64_t e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
        for (int64_t e = e0; e < e1; ++e) {
          const int32_t code = a.tcf[e];
          const int lf = code >> 1;
          const T sa = (code & 1) ? -a.cf[e].area : a.cf[e].area;
#pragma unroll
          for (int r = 0; r < NR; ++r) flux[r] += sa * sPhi[(size_t(lf) * NR + r) * BV + lane];
        }
        const T inv_vol = T(1.0 / a.vol[c]);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const size_t idx = frow(r, m, c, M, Nc) + lane;
          const T f = a.f_cur[idx];
          const T ft = f - flux[r] * inv_vol + beta0 * (fp[r] - f);
          a.f_next[idx] = real_v ? ft : T(0);
        }
      }
      // no barrier here: the next tile's phase G writes only sG, which phase S
      // does not read; the barrier after that phase G orders sPhi
    }
  }
  __syncthreads();

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t c0 = a.tile_begin[tile], c1 = a.tile_begin[tile + 1];
    const int nt = int(c1 - c0);
    const TileFace* tf = a.tf + a.tf_off[tile];
    const int nfc = int(a.tf_off[tile + 1] - a.tf_off[tile]);
    double* Facc = a.Facc + size_t(tile) * a.Facc_stride;

    // ---- wall density from non-penetration (Eq. 38), completed wall fluxes ----
    for (int lf = threadIdx.x; lf < nfc; lf += blockDim.x) {
      const FaceGeom<T>& fg = a.fg[tf[lf].face];
      if (fg.bc_type != 1) continue;
      double* F = Facc + size_t(lf) * FACC_W;
      const double rw = F[5] != 0.0 ? -F[0] / F[5] : 0.0;
      for (int t = 0; t < NW; ++t) F[t] += rw * F[5 + t];
      F[10] = rw;
    }
    __syncthreads();

    // ---- conservative update (Eq. 27) and the W^{n+1} primitive record ----
    __shared__ double s_res[32][NWP];
    double res[NWP] = {0, 0, 0, 0, 0};
    for (int li = threadIdx.x; li < nt; li += blockDim.x) {
      const int64_t c = c0 + li;
      double acc[NWP] = {0, 0, 0, 0, 0};
      for (int64_t e = a.cf_off[c]; e < a.cf_off[c + 1]; ++e) {
        const int32_t code = a.tcf[e];
        const int lf = code >> 1;
        const double sa = (code & 1) ? -double(a.cf[e].area) : double(a.cf[e].area);
        const double* F = Facc + size_t(lf) * FACC_W;
#pragma unroll
        for (int t = 0; t < NW; ++t) acc[t] += sa * F[t];
      }
      const double iv = 1.0 / a.vol[c];
      double Wn[NWP];
#pragma unroll
      for (int t = 0; t < NW; ++t) {
        const double w0 = a.W_cur[c * NWP + t];
        Wn[t] = w0 - acc[t] * iv;
        a.W_next[c * NWP + t] = Wn[t];
        res[t] += (Wn[t] - w0) * (Wn[t] - w0);
      }
      CellPrim pn;
      double u2 = 0.0;
      pn.rho = Wn[0];
#pragma unroll
      for (int d = 0; d < 3; ++d) pn.U[d] = d < D ? Wn[1 + (d < D ? d : 0)] / Wn[0] : 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) u2 += pn.U[d] * pn.U[d];
      const double ein = Wn[D + 1] - 0.5 * Wn[0] * u2;
      pn.lam = (a.g.K + 3) * Wn[0] / (4.0 * ein);
      const bool ok = (pn.rho > 0.0) && (ein > 0.0) && isfinite(pn.lam) && isfinite(u2);
      if (!ok) {
        atomicOr(a.status, 1);
        pn.rho = 1.0;
        pn.lam = 1.0;
      }
      pn.tau = a.g.mu_ref * pow(1.0 / pn.lam, a.g.omega) * 2.0 * pn.lam / pn.rho;
#pragma unroll
      for (int d = 0; d < 3; ++d) pn.q[d] = a.cp[c].q[d];  // lagged heat flux in stage 2
      pn.pad = 0.0;
      a.cp_next[c] = pn;
    }
#pragma unroll
    for (int t = 0; t < NW; ++t) res[t] = warp_sum(res[t]);
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < NW; ++t) s_res[warp][t] = res[t];
    __syncthreads();
    if (threadIdx.x < NW) {
      double sum = 0.0;
      for (int w_ = 0; w_ < nwarps; ++w_) sum += s_res[w_][threadIdx.x];
      atomicAdd(a.res_acc + threadIdx.x, sum);
    }

    // ---- second stage (Eq. 42) and the heat flux of f^{n+1} (Eq. 13) ----
    for (int li = warp; li < nt; li += nwarps) {
      const int64_t c = c0 + li;
      const CellPrim& p = a.cp_next[c];
      const T rho = T(p.rho), lam = T(p.lam), beta1 = dt / (T(2) * T(p.tau));
      const T inv1 = T(1) / (T(1) + beta1);
      const T pref = rho * maxwell_pref<D>(lam);
      const T s0 = a.g.shakhov ? T(4.0 * (1.0 - a.g.Pr)) * lam * lam / (T(5) * rho) : T(0);
      const T kap = T(Kxi) / (T(2) * lam);
      const T iv = T(1.0 / a.vol[c]);
      const int64_t e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
      bool has_wall = false;
      for (int64_t e = e0; e < e1; ++e) has_wall |= (a.cf[e].flags & 1) != 0;
      double qacc[3] = {0.0, 0.0, 0.0};
      for (int64_t m = 0; m < M; ++m) {
        const int64_t k = m * BV + lane;
        T u[3];
        u[0] = a.ux[k];
        u[1] = D > 1 ? a.uy[k] : T(0);
        u[2] = D > 2 ? a.uz[k] : T(0);
        const bool real_v = k < a.nv;
        T ft[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) ft[r] = a.f_next[frow(r, m, c, M, Nc) + lane];
        if (has_wall) {
          // outgoing wall flux rho_w G_w for u.n < 0, known only after the sweep
          for (int64_t e = e0; e < e1; ++e) {
            if (!(a.cf[e].flags & 1)) continue;
            const int lf = a.tcf[e] >> 1;
            const int64_t fidx = tf[lf].face;
            const FaceGeom<T>& fg = a.fg[fidx];
            const FaceRec<T>& R = a.fr[fidx];
            T un = T(0), c2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              un += u[d] * fg.n[d];
              c2 += (u[d] - R.U[d]) * (u[d] - R.U[d]);
            }
            if (un < T(0)) {
              const T rw = T(Facc[size_t(lf) * FACC_W + 10]);
              const T out = un * dt * rw * R.rho_pref * t_exp(-R.lam * c2);
              ft[0] -= a.cf[e].area * iv * out;
              if (NR == 2) ft[NR - 1] -= a.cf[e].area * iv * R.kappa * out;
            }
          }
        }
        T cc[3], c2 = T(0), cq = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          cc[d] = u[d] - T(p.U[d]);
          c2 += cc[d] * cc[d];
          cq += cc[d] * T(p.q[d]);
        }
        const T H = pref * t_exp(-lam * c2);
        const T s = s0 * cq;
        T f1[NR];
        f1[0] = (ft[0] + beta1 * H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)))) * inv1;
        if (NR == 2) f1[NR - 1] = (ft[NR - 1] + beta1 * kap * H * (T(1) + s * (T(2) * lam * c2 - T(D)))) * inv1;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (!real_v) f1[r] = T(0);
          a.f_next[frow(r, m, c, M, Nc) + lane] = f1[r];
        }
        const T wq = real_v ? T(0.5) * a.w[k] : T(0);
        const T e_ = c2 * f1[0] + (NR == 2 ? f1[NR - 1] : T(0));
        const T qs = warp_sum8<T>(wq * cc[0] * e_, D > 1 ? wq * cc[1] * e_ : T(0), D > 2 ? wq * cc[2] * e_ : T(0),
                                  T(0), T(0), T(0), T(0), T(0), lane);
        if (writer8 && idx8 < D) qacc[idx8 == 0 ? 0 : idx8 == 1 ? 1 : 2] += double(qs);
      }
      if (writer8 && idx8 < D) a.q_next[c * 3 + idx8] = idx8 == 0 ? qacc[0] : idx8 == 1 ? qacc[1] : qacc[2];
    }
    __syncthreads();
  }
}

template <int D, int NR, typename T>
static cudaError_t launch_tpl(cudaStream_t s, const SweepArgs<T>& a, int grid, int threads, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep<D, NR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k_sweep<D, NR, T><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep(cudaStream_t s, const SweepArgs<T>& a, int grid, int threads, size_t smem) {
  const int D = a.g.D, NR = a.g.NR;
  if (D == 1 && NR == 2) return launch_tpl<1, 2, T>(s, a, grid, threads, smem);
  if (D == 2 && NR == 2) return launch_tpl<2, 2, T>(s, a, grid, threads, smem);
  if (D == 3 && NR == 1) return launch_tpl<3, 1, T>(s, a, grid, threads, smem);
  if (D == 3 && NR == 2) return launch_tpl<3, 2, T>(s, a, grid, threads, smem);
  return cudaErrorInvalidValue;
}

template <int D, int NR, typename T>
static int occ_tpl(int threads, size_t smem) {
  int n = 0;
  if (cudaFuncSetAttribute(k_sweep<D, NR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<D, NR, T>, threads, smem) != cudaSuccess) return 0;
  return n;
}

template <typename T>
int sweep_occupancy(int D, int NR, int threads, size_t smem) {
  if (D == 1 && NR == 2) return occ_tpl<1, 2, T>(threads, smem);
  if (D == 2 && NR == 2) return occ_tpl<2, 2, T>(threads, smem);
  if (D == 3 && NR == 1) return occ_tpl<3, 1, T>(threads, smem);
  if (D == 3 && NR == 2) return occ_tpl<3, 2, T>(threads, smem);
  return 0;
}

// ---------------------------------------------------------------------------
// Scratch of the allocation-free step (ugks_step_static_scratch).  Every GPU
// that loads this library holds this array until the process exits.  In host
// code the symbol is only a host-side stand-in: its device address must be
// obtained with cudaGetSymbolAddress, once per device, with that device
// current; kernels receive that address.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_sweep_scratch[kStaticScratchBytes];

cudaError_t static_scratch_address(void** ptr) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_sweep_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

template cudaError_t launch_sweep<float>(cudaStream_t, const SweepArgs<float>&, int, int, size_t);
template cudaError_t launch_sweep<double>(cudaStream_t, const SweepArgs<double>&, int, int, size_t);
template int sweep_occupancy<float>(int, int, int, size_t);
template int sweep_occupancy<double>(int, int, int, size_t);

}  // namespace ugks
