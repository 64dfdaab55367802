// Per-query epilogue of the fused lnL kernels: extrinsic amplitudes, spline
// stencil at each detector delay, SVD-basis reconstruction of the overlaps and
// the Hermitian cross-term form.  Shared by the FP32 SIMT kernel and the
// tcgen05 kernels; the caller supplies an accessor that loads 8 consecutive
// interpolated columns of this query's row.
#pragma once

#include "mf_internal.cuh"

namespace mf {

// Read-only global loads with L1 policies: table entries stream through
// (no L1 allocation) so that they do not evict the node coordinates, which
// every k-block of every tile re-reads (kept with evict_last).
__device__ __forceinline__ float4 ldg_stream(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ldg_keep(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// -2Y_lm(iota, phi) = A(iota) e^{i m phi}.  Closed forms in
// c2 = cos^2(iota/2), s2 = sin^2(iota/2), cs = cos(iota/2) sin(iota/2),
// obtained from the Wigner-d representation of spin-weighted harmonics
// (Eq. h_spherical_harmonic_basis); Ap is the +m amplitude, Am the -m one.
__device__ __forceinline__ void ylm_amps(int l, int m, float c2, float s2, float cs,
                                         float &Ap, float &Am) {
    const float k22 = 0.63078313050504f;   // sqrt(5)/(2 sqrt(pi))
    const float k21 = 1.26156626101008f;   // sqrt(5)/sqrt(pi)
    const float k33 = 1.82818319785786f;   // sqrt(42)/(2 sqrt(pi))
    const float k32 = 0.74635266518023f;   // sqrt(7)/(2 sqrt(pi))
    const float k44 = 4.47811599108140f;   // 3 sqrt(7)/sqrt(pi)
    switch (l * 10 + m) {
        case 22: Ap = k22 * c2 * c2; Am = k22 * s2 * s2; break;
        case 21: Ap = k21 * c2 * cs; Am = k21 * s2 * cs; break;
        case 33: Ap = -k33 * c2 * c2 * cs; Am = k33 * s2 * s2 * cs; break;
        case 32: Ap = k32 * c2 * c2 * (c2 - 5.f * s2); Am = k32 * s2 * s2 * (5.f * c2 - s2); break;
        case 44: Ap = k44 * c2 * c2 * cs * cs; Am = k44 * s2 * s2 * cs * cs; break;
        default: Ap = 0.f; Am = 0.f; break;
    }
}

struct QueryExt {
    float a;            // d_ref / d_L
    float c2, s2, cs;   // half-angle combinations of iota
    float c2p, s2p;     // cos 2psi, sin 2psi
    float cph, sph;     // cos phi_c, sin phi_c
    float tc;
    float alpha, sd, cd;   // sky mode: right ascension, sin and cos of the declination
};

__device__ __forceinline__ QueryExt load_ext(const EpiParams &P, const float *ext, int E, int q) {
    const float *e = ext + (size_t)q * E;
    QueryExt x;
    float dL = e[0], ci = e[1], psi = e[2], phc = e[3];
    x.tc = e[4];
    x.a = P.d_ref / dL;
    ci = fminf(1.f, fmaxf(-1.f, ci));
    x.c2 = 0.5f * (1.f + ci);
    x.s2 = 0.5f * (1.f - ci);
    x.cs = 0.5f * sqrtf(fmaxf(0.f, (1.f - ci) * (1.f + ci)));
    sincosf(2.f * psi, &x.s2p, &x.c2p);
    sincosf(phc, &x.sph, &x.cph);
    x.alpha = 0.f;
    x.sd = 0.f;
    x.cd = 1.f;
    if (P.sky) {
        x.alpha = e[5];
        sincosf(e[6], &x.sd, &x.cd);
    }
    return x;
}

// Antenna patterns (F+, Fx) of detector k at the query's polarisation angle
// and its geocentre-to-detector delay dt (Eqs. projected_h_td/fd).  Frozen
// patterns: F(psi) = rotation of (F+0, Fx0) by 2 psi, the delay is in the
// detector's sample offset (dt = 0 here).  Sky mode: with the hour angle
// h = gk + omega t_c - alpha, the source direction w = (cos d cos h,
// -cos d sin h, sin d) and the wave-frame axes at psi = 0, X0 = (-sin h,
// -cos h, 0), Y0 = (-cos h sin d, sin h sin d, cos d), the detector tensor D
// gives F+0 = X0.D.X0 - Y0.D.Y0 and Fx0 = 2 X0.D.Y0, which rotate with 2 psi
// like the frozen ones; dt = -(r . w), r = position / c.
__device__ __forceinline__ void det_response(const EpiParams &P, int k, const QueryExt &x, float &fp,
                                             float &fx, float &dt) {
    float fp0 = P.fp0[k], fx0 = P.fx0[k];
    dt = 0.f;
    if (P.sky) {
        float sh, ch;
        sincosf(P.gk[k] + P.omega * x.tc - x.alpha, &sh, &ch);
        const float X[3] = {-sh, -ch, 0.f};
        const float Y[3] = {-ch * x.sd, sh * x.sd, x.cd};
        const float *D = P.dten[k];
        // a.D.b for the symmetric D stored as (xx, yy, zz, xy, xz, yz)
        auto quad = [&](const float (&a)[3], const float (&b)[3]) {
            return D[0] * a[0] * b[0] + D[1] * a[1] * b[1] + D[2] * a[2] * b[2] +
                   D[3] * (a[0] * b[1] + a[1] * b[0]) + D[4] * (a[0] * b[2] + a[2] * b[0]) +
                   D[5] * (a[1] * b[2] + a[2] * b[1]);
        };
        fp0 = quad(X, X) - quad(Y, Y);
        fx0 = 2.f * quad(X, Y);
        dt = -(P.dpos[k][0] * x.cd * ch - P.dpos[k][1] * x.cd * sh + P.dpos[k][2] * x.sd);
    }
    fp = fp0 * x.c2p + fx0 * x.s2p;
    fx = -fp0 * x.s2p + fx0 * x.c2p;
}

// c_k,mu = (d_ref/d_L)/2 e^{-i m phi_c} [F+ (A- + (-1)^l A+) + i Fx (A- - (-1)^l A+)]
// (Eqs. hplus_hcross_decomposed1/2 in Eq. projected_h_fd), for the detector's
// antenna patterns (fp, fx) at the query's polarisation angle.
template <int NM>
__device__ __forceinline__ void det_amplitudes(const EpiParams &P, float fp, float fx, const QueryExt &x,
                                               float (&cre)[NM], float (&cim)[NM]) {
#pragma unroll
    for (int mu = 0; mu < NM; ++mu) {
        int l = P.ell[mu], m = P.em[mu];
        float Ap, Am;
        ylm_amps(l, m, x.c2, x.s2, x.cs, Ap, Am);
        float sg = (l & 1) ? -1.f : 1.f;
        float re = 0.5f * x.a * fp * (Am + sg * Ap);
        float im = 0.5f * x.a * fx * (Am - sg * Ap);
        // multiply by e^{-i m phi}
        float er = 1.f, ei = 0.f;
        for (int t = 0; t < m; ++t) {
            float nr = er * x.cph + ei * x.sph;
            float ni = ei * x.cph - er * x.sph;
            er = nr; ei = ni;
        }
        cre[mu] = re * er - im * ei;
        cim[mu] = re * ei + im * er;
    }
}

// Spline interval for detector k: sample j with t_c + dt_k in [t_j, t_j+1)
// and the offset u in [0,1) (dt: the sky-dependent part of the delay, 0 for
// frozen patterns).  Returns false when the 10-sample window j-4..j+5 leaves
// [0, M) (j is then clamped so that reads stay in range).
__device__ __forceinline__ bool det_interval(const EpiParams &P, int k, float tc, float dt, int &j,
                                             float &u) {
    float v = fmaf(tc + dt, P.inv_dt, P.frac[k]);
    if (!(fabsf(v) < 1.0e7f)) {   // NaN / absurd times
        j = kStencilLo;
        u = 0.f;
        return false;
    }
    float fl = floorf(v);
    u = v - fl;
    j = P.J[k] + (int)fl;
    bool ok = (j - kStencilLo >= 0) && (j - kStencilLo + kStencil <= P.M);
    if (!ok) j = kStencilLo;
    return ok;
}

// lnL contribution of the groups of one pass for one query.  Acc provides
//   __device__ void load8(int col, float (&f)[8]);
// returning columns [col, col+8) of this query's row of the pass.
template <int NM, class Acc>
__device__ __forceinline__ float pass_lnl(const EpiParams &P, const Pass &ps, const QueryExt &x,
                                          Acc &acc, bool &bad) {
    float lnl = 0.f;
    int cur = -1, j = 0;
    float u = 0.f;
    float cre[NM], cim[NM];
    for (int g = ps.g0; g < ps.g0 + ps.ng; ++g) {
        const Group G = P.groups[g];
        if (G.det != cur) {
            cur = G.det;
            // control flow stays warp-uniform (the tcgen05 accessor loads with
            // .sync.aligned): an out-of-window query reads an in-range
            // interval and is flagged instead of skipped
            float fp, fx, dt;
            det_response(P, cur, x, fp, fx, dt);
            if (!det_interval(P, cur, x.tc, dt, j, u)) bad = true;
            det_amplitudes<NM>(P, fp, fx, x, cre, cim);
        }
        if (G.kind == 0) {
            // Eq. (SVD) at t_c + dt_k: z = sum_i C_i S_i(u), S_i the spline of
            // basis vector i on interval j (cubic in u from the table)
            // this group's coefficients [G.i0, G.i0 + G.ni) of the mode
            const float4 *tp = P.cubic + (((size_t)(G.det * P.n_modes + G.mode) * P.M + j) * P.rank + G.i0) * 2;
            const int ni = G.ni;
            float zr = 0.f, zi = 0.f;
            // table entries of the next 4 coefficients are loaded one chunk
            // ahead so their latency overlaps the current chunk's math
            float4 cur[8], nxt[8];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool in = t < ni;
                cur[2 * t] = in ? ldg_stream(tp + 2 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
                cur[2 * t + 1] = in ? ldg_stream(tp + 2 * t + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            for (int i0 = 0; i0 < ni; i0 += 4) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool in = i0 + 4 + t < ni;
                    nxt[2 * t] = in ? ldg_stream(tp + 2 * (i0 + 4 + t)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    nxt[2 * t + 1] = in ? ldg_stream(tp + 2 * (i0 + 4 + t) + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                float f[8];
                acc.load8(G.col + 2 * i0, f);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float4 c01 = cur[2 * t], c23 = cur[2 * t + 1];
                    float br = fmaf(u, fmaf(u, fmaf(u, c23.z, c23.x), c01.z), c01.x);
                    float bi = fmaf(u, fmaf(u, fmaf(u, c23.w, c23.y), c01.w), c01.y);
                    // columns beyond the rank are zero padding (their f are 0)
                    zr = fmaf(f[2 * t], br, fmaf(-f[2 * t + 1], bi, zr));
                    zi = fmaf(f[2 * t], bi, fmaf(f[2 * t + 1], br, zi));
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) cur[t] = nxt[t];
            }
            float mr = 0.f, mi = 0.f;
#pragma unroll
            for (int mu = 0; mu < NM; ++mu)
                if (mu == G.mode) { mr = cre[mu]; mi = cim[mu]; }
            lnl += mr * zr + mi * zi;
        } else {
            constexpr int NS = NM * NM;
            constexpr int NL = (NS + 7) / 8;
            float f[NL * 8];
#pragma unroll
            for (int c = 0; c < NL; ++c) {
                float t8[8];
                acc.load8(G.col + 8 * c, t8);
#pragma unroll
                for (int e = 0; e < 8; ++e) f[8 * c + e] = t8[e];
            }
            float quad = 0.f;
#pragma unroll
            for (int mu = 0; mu < NM; ++mu) quad += (cre[mu] * cre[mu] + cim[mu] * cim[mu]) * f[mu];
            int p = NM;
#pragma unroll
            for (int mu = 0; mu < NM; ++mu)
#pragma unroll
                for (int nu = mu + 1; nu < NM; ++nu) {
                    float xr = cre[mu] * cre[nu] + cim[mu] * cim[nu];
                    float xi = cre[mu] * cim[nu] - cim[mu] * cre[nu];
                    quad += 2.f * (xr * f[p] - xi * f[p + 1]);
                    p += 2;
                }
            lnl -= 0.5f * quad;
        }
    }
    return lnl;
}

// Interpolated columns of one pass for one query: the Phi.W stage alone
// (Eq. rbfcoeff), scattered into the query's row of out [Q][K] in the
// node_values column order; padding columns (user column -1) are dropped.
// The loop is warp-uniform (the tcgen05 accessor loads are warp-collective);
// row == nullptr (a query past the batch) loads without storing.
template <class Acc>
__device__ __forceinline__ void pass_columns(const Pass &ps, Acc &acc, const int *__restrict__ user_of_dev,
                                             float *row) {
    for (int c = 0; c < ps.width; c += 8) {
        float f[8];
        acc.load8(c, f);
        if (row) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int u = __ldg(user_of_dev + ps.col0 + c + e);
                if (u >= 0) row[u] = f[e];
            }
        }
    }
}

}  // namespace mf
