// FP64 kernels around the convolution: Green-kernel tabulation and spectra (eqs. 5, 7, 10 and the
// equal-volume-sphere self term of Section 2.2), the contrast upload (Section 2.1), the incident
// field of a magnetic dipole, and the receiver fields of eq. 4.
#include "green.cuh"

namespace ie {

// e^{ikR} for complex k = (kr, ki): e^{-ki R} (cos kr R, sin kr R)
__device__ __forceinline__ double2 expikr(double2 k, double R) {
  double s, c;
  sincos(k.x * R, &s, &c);
  const double a = exp(-k.y * R);
  return make_double2(a * c, a * s);
}

// One component of dv * G^E(R) (eq. 5 differentiated in closed form):
//   G^E_pq = (g / sigma0) [ (k^2 + (ikR - 1)/R^2) delta_pq + (3 - 3ikR - k^2 R^2)/R^2 Rhat_p Rhat_q ]
// using i omega mu0 = k^2 / sigma0. comp: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz.
__device__ double2 green_component(int comp, double rx, double ry, double rz, double2 k, double sigma0,
                                   double dv) {
  const double R2 = rx * rx + ry * ry + rz * rz, R = sqrt(R2);
  const double2 e = expikr(k, R);
  const double gs = dv / (4.0 * M_PI * R * sigma0);
  const double2 g = make_double2(gs * e.x, gs * e.y);  // dv g / sigma0
  const double2 k2 = make_double2(k.x * k.x - k.y * k.y, 2.0 * k.x * k.y);
  const double2 ikR = make_double2(-k.y * R, k.x * R);
  // a = k^2 + (ikR - 1)/R^2 ; b = (3 - 3ikR - k^2 R^2)/R^2
  const double2 a = make_double2(k2.x + (ikR.x - 1.0) / R2, k2.y + ikR.y / R2);
  const double2 b = make_double2((3.0 - 3.0 * ikR.x) / R2 - k2.x, (-3.0 * ikR.y) / R2 - k2.y);
  const double ux = rx / R, uy = ry / R, uz = rz / R;
  double d, q;
  switch (comp) {
    case 0: d = 1; q = ux * ux; break;
    case 1: d = 1; q = uy * uy; break;
    case 2: d = 1; q = uz * uz; break;
    case 3: d = 0; q = ux * uy; break;
    case 4: d = 0; q = ux * uz; break;
    default: d = 0; q = uy * uz; break;
  }
  const double2 s = make_double2(d * a.x + q * b.x, d * a.y + q * b.y);
  return cmul(g, s);
}

// Circulant embedding along one axis of length L for a grid of n cells: index m holds offset m for
// m <= n-1, offset m-L for m >= L-(n-1), and nothing (flag false) otherwise.
__device__ __forceinline__ bool embed(int m, int n, int L, int* d) {
  if (m <= n - 1) { *d = m; return true; }
  if (m >= L - (n - 1)) { *d = m - L; return true; }
  return false;
}

__global__ void k_green_tab(double2* __restrict__ out, int comp, int Lx, int Ly, int Lz, int nx, int ny, int nz,
                            double h, double2 k, double sigma0, double2 self) {
  const long total = (long)Lx * Ly * Lz;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int mx = (int)(idx % Lx), my = (int)((idx / Lx) % Ly), mz = (int)(idx / ((long)Lx * Ly));
    int dx, dy, dz;
    double2 v = make_double2(0.0, 0.0);
    if (embed(mx, nx, Lx, &dx) && embed(my, ny, Ly, &dy) && embed(mz, nz, Lz, &dz)) {
      if (dx == 0 && dy == 0 && dz == 0) {
        if (comp < 3) v = self;
      } else {
        v = green_component(comp, dx * h, dy * h, dz * h, k, sigma0, h * h * h);
      }
    }
    out[idx] = v;
  }
}

__global__ void k_extract_octant(const double2* __restrict__ full, int Lx, int Ly, int Lz, double scale,
                                 double2* __restrict__ o64, float2* __restrict__ o32, float4* __restrict__ odf) {
  const int ox = Lx / 2 + 1, oy = Ly / 2 + 1, oz = Lz / 2 + 1;
  const long total = (long)ox * oy * oz;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % ox), iy = (int)((idx / ox) % oy), iz = (int)(idx / ((long)ox * oy));
    const double2 v = full[((long)iz * Ly + iy) * Lx + ix];
    const double2 s = make_double2(scale * v.x, scale * v.y);
    o64[idx] = s;
    o32[idx] = make_float2((float)s.x, (float)s.y);
    const df re(s.x), im(s.y);
    odf[idx] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// sigma6 [N][6] (absolute, xx yy zz xy xz yz) -> dsigma [6][N] = sigma - sigma0 I in f64 and f32.
// Sets *bad when a value is not finite or sigma is not positive definite (leading minors).
__global__ void k_set_contrast(const double* __restrict__ s6, long N, double sigma0, double* __restrict__ d64,
                               float* __restrict__ d32, int* __restrict__ bad) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    double s[6];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      s[c] = s6[i * 6 + c];
      ok = ok && isfinite(s[c]);
    }
    const double m1 = s[0], m2 = s[0] * s[1] - s[3] * s[3];
    const double det = s[0] * (s[1] * s[2] - s[5] * s[5]) - s[3] * (s[3] * s[2] - s[5] * s[4]) +
                       s[4] * (s[3] * s[5] - s[1] * s[4]);
    ok = ok && m1 > 0.0 && m2 > 0.0 && det > 0.0;
    if (!ok) atomicOr(bad, 1);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double v = s[c] - (c < 3 ? sigma0 : 0.0);
      d64[c * N + i] = v;
      d32[c * N + i] = (float)v;
    }
  }
}

// act[z] = 1 if any contrast component of plane z is non-zero (one block per plane).
__global__ void k_plane_active(const double* __restrict__ d64, long N, long nxy, int* __restrict__ act) {
  const long z = blockIdx.x;
  int any = 0;
  for (long i = threadIdx.x; i < nxy && !any; i += blockDim.x) {
    const long o = z * nxy + i;
#pragma unroll
    for (int c = 0; c < 6; ++c) any |= (d64[c * N + o] != 0.0);
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) act[z] = any;
}

// Contraction-form tensors from the contrast (both symmetric, [6][N], FP64 and FP32):
//   M = 2 sigma0 (sigma + sigma0 I)^-1 = 2 sigma0 (dsigma + 2 sigma0 I)^-1,   K = dsigma M
// (dsigma and M commute, so K is symmetric). The inverse is the adjugate over the determinant of the
// positive definite sigma + sigma0 I.
__global__ void k_contract_tensors(const double* __restrict__ d64, long N, double sigma0, double* __restrict__ K64,
                                   double* __restrict__ M64, float* __restrict__ K32, float* __restrict__ M32) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double dxx = d64[i], dyy = d64[N + i], dzz = d64[2 * N + i];
    const double dxy = d64[3 * N + i], dxz = d64[4 * N + i], dyz = d64[5 * N + i];
    const double axx = dxx + 2 * sigma0, ayy = dyy + 2 * sigma0, azz = dzz + 2 * sigma0;
    const double cxx = ayy * azz - dyz * dyz, cyy = axx * azz - dxz * dxz, czz = axx * ayy - dxy * dxy;
    const double cxy = dxz * dyz - dxy * azz, cxz = dxy * dyz - dxz * ayy, cyz = dxy * dxz - axx * dyz;
    const double det = axx * cxx + dxy * cxy + dxz * cxz;
    const double f = 2 * sigma0 / det;
    const double m[6] = {f * cxx, f * cyy, f * czz, f * cxy, f * cxz, f * cyz};
    // K = dsigma M (symmetric): rows of dsigma times columns of M
    const double k[6] = {dxx * m[0] + dxy * m[3] + dxz * m[4], dxy * m[3] + dyy * m[1] + dyz * m[5],
                         dxz * m[4] + dyz * m[5] + dzz * m[2], dxx * m[3] + dxy * m[1] + dxz * m[5],
                         dxx * m[4] + dxy * m[5] + dxz * m[2], dxy * m[4] + dyy * m[5] + dyz * m[2]};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      M64[c * N + i] = m[c];
      K64[c * N + i] = k[c];
      M32[c * N + i] = (float)m[c];
      K32[c * N + i] = (float)k[c];
    }
  }
}

// x := M x in place for a symmetric [6][...] tensor (block-local vectors, component stride cs).
template <typename V, typename R>
__global__ void k_apply_sym6(const R* __restrict__ M, long m_cs, V* __restrict__ x, long cs, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const R mxx = M[i], myy = M[m_cs + i], mzz = M[2 * m_cs + i], mxy = M[3 * m_cs + i], mxz = M[4 * m_cs + i],
            myz = M[5 * m_cs + i];
    const V a = x[i], b = x[cs + i], c = x[2 * cs + i];
    V o0, o1, o2;
    o0.x = mxx * a.x + mxy * b.x + mxz * c.x;
    o0.y = mxx * a.y + mxy * b.y + mxz * c.y;
    o1.x = mxy * a.x + myy * b.x + myz * c.x;
    o1.y = mxy * a.y + myy * b.y + myz * c.y;
    o2.x = mxz * a.x + myz * b.x + mzz * c.x;
    o2.y = mxz * a.y + myz * b.y + mzz * c.y;
    x[i] = o0;
    x[cs + i] = o1;
    x[2 * cs + i] = o2;
  }
}

// Incident field E0 = i omega mu0 grad g(r - r_s) x m at every cell centre, c128 [3][N].
__global__ void k_incident_E(double2* __restrict__ E0, int nx, int ny, int nz, double ox, double oy, double oz,
                             double h, double sx, double sy, double sz, double mx, double my, double mz, double2 k,
                             double omega_mu0) {
  const long N = (long)nx * ny * nz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long)nx * ny));
    const double rx = ox + (ix + 0.5) * h - sx, ry = oy + (iy + 0.5) * h - sy, rz = oz + (iz + 0.5) * h - sz;
    const double R = sqrt(rx * rx + ry * ry + rz * rz);
    const double2 e = expikr(k, R);
    // grad g = g (ik - 1/R) Rvec / R ; f = g (ik - 1/R) / R
    const double gs = 1.0 / (4.0 * M_PI * R);
    const double2 g = make_double2(gs * e.x, gs * e.y);
    const double2 f0 = make_double2(-k.y - 1.0 / R, k.x);
    const double2 f = cmul(g, make_double2(f0.x / R, f0.y / R));
    // (grad g x m) = f (Rvec x m); times i omega mu0
    const double cx = ry * mz - rz * my, cy = rz * mx - rx * mz, cz = rx * my - ry * mx;
    const double2 iw = make_double2(-omega_mu0 * f.y, omega_mu0 * f.x);  // i omega mu0 f
    E0[i] = make_double2(iw.x * cx, iw.y * cx);
    E0[N + i] = make_double2(iw.x * cy, iw.y * cy);
    E0[2 * N + i] = make_double2(iw.x * cz, iw.y * cz);
  }
}

// Scattered magnetic field partial sums: H^s(r_r) = sum_j dv grad g(r_r - r_j) x (dsigma_j E_j).
// part[(blk * n_rx + r) * 3 + c]
__global__ void __launch_bounds__(256) k_receivers(const double2* __restrict__ E, long e_cs, const double* __restrict__ ds,
                                                   long N, int nx, int ny, double ox, double oy, double oz, double h,
                                                   const double* __restrict__ rx, int n_rx, double2 k,
                                                   double2* __restrict__ part) {
  __shared__ double2 red[kMaxRx * 3][8];
  double2 acc[kMaxRx * 3];
#pragma unroll
  for (int q = 0; q < kMaxRx * 3; ++q) acc[q] = make_double2(0.0, 0.0);
  const double dv = h * h * h;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long)nx * ny));
    const double cx = ox + (ix + 0.5) * h, cy = oy + (iy + 0.5) * h, cz = oz + (iz + 0.5) * h;
    const double2 e0 = E[i], e1 = E[e_cs + i], e2 = E[2 * e_cs + i];
    const double sxx = ds[i], syy = ds[N + i], szz = ds[2 * N + i], sxy = ds[3 * N + i], sxz = ds[4 * N + i],
                 syz = ds[5 * N + i];
    const double2 J0 = make_double2(sxx * e0.x + sxy * e1.x + sxz * e2.x, sxx * e0.y + sxy * e1.y + sxz * e2.y);
    const double2 J1 = make_double2(sxy * e0.x + syy * e1.x + syz * e2.x, sxy * e0.y + syy * e1.y + syz * e2.y);
    const double2 J2 = make_double2(sxz * e0.x + syz * e1.x + szz * e2.x, sxz * e0.y + syz * e1.y + szz * e2.y);
    if (J0.x == 0.0 && J0.y == 0.0 && J1.x == 0.0 && J1.y == 0.0 && J2.x == 0.0 && J2.y == 0.0) continue;
#pragma unroll
    for (int r = 0; r < kMaxRx; ++r) {
      if (r < n_rx) {
        const double Rx = rx[3 * r] - cx, Ry = rx[3 * r + 1] - cy, Rz = rx[3 * r + 2] - cz;
        const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
        const double2 e = expikr(k, R);
        const double gs = dv / (4.0 * M_PI * R * R);
        const double2 f = cmul(make_double2(gs * e.x, gs * e.y), make_double2(-k.y - 1.0 / R, k.x));
        // dv grad g = f Rvec ; (Rvec x J)
        const double2 X = make_double2(Ry * J2.x - Rz * J1.x, Ry * J2.y - Rz * J1.y);
        const double2 Y = make_double2(Rz * J0.x - Rx * J2.x, Rz * J0.y - Rx * J2.y);
        const double2 Z = make_double2(Rx * J1.x - Ry * J0.x, Rx * J1.y - Ry * J0.y);
        acc[3 * r] = acc[3 * r] + cmul(f, X);
        acc[3 * r + 1] = acc[3 * r + 1] + cmul(f, Y);
        acc[3 * r + 2] = acc[3 * r + 2] + cmul(f, Z);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxRx * 3; ++q) {
    double2 v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < n_rx * 3) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + red[threadIdx.x][w];
    part[(long)blockIdx.x * n_rx * 3 + threadIdx.x] = s;
  }
}

// Sum the per-block partials and add the incident field H0 = (k^2 g I + grad grad g) m of the source.
__global__ void k_receivers_finish(const double2* __restrict__ part, int nblk, const double* __restrict__ rx,
                                   int n_rx, double sx, double sy, double sz, double mx, double my, double mz,
                                   double2 k, double2* __restrict__ H) {
  const int q = threadIdx.x;
  if (q >= n_rx * 3) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = s + part[(long)b * n_rx * 3 + q];
  const int r = q / 3, c = q % 3;
  const double Rx = rx[3 * r] - sx, Ry = rx[3 * r + 1] - sy, Rz = rx[3 * r + 2] - sz;
  const double R2 = Rx * Rx + Ry * Ry + Rz * Rz, R = sqrt(R2);
  const double2 e = expikr(k, R);
  const double gs = 1.0 / (4.0 * M_PI * R);
  const double2 g = make_double2(gs * e.x, gs * e.y);
  const double2 k2 = make_double2(k.x * k.x - k.y * k.y, 2.0 * k.x * k.y);
  const double2 ikR = make_double2(-k.y * R, k.x * R);
  const double2 a = cmul(g, make_double2(k2.x + (ikR.x - 1.0) / R2, k2.y + ikR.y / R2));
  const double2 b = cmul(g, make_double2((3.0 - 3.0 * ikR.x) / R2 - k2.x, (-3.0 * ikR.y) / R2 - k2.y));
  const double u[3] = {Rx / R, Ry / R, Rz / R}, m[3] = {mx, my, mz};
  const double um = u[0] * m[0] + u[1] * m[1] + u[2] * m[2];
  const double2 h0 = make_double2(a.x * m[c] + b.x * u[c] * um, a.y * m[c] + b.y * u[c] * um);
  H[q] = s + h0;
}

// ------------------------------------------------------------------------------------------- launchers
static inline unsigned grid_for(long n, int threads, int cap) {
  long g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

cudaError_t launch_green_tab(double2* out, int comp, int Lx, int Ly, int Lz, int nx, int ny, int nz, double h,
                             double2 k, double sigma0, double2 self, cudaStream_t s) {
  k_green_tab<<<grid_for((long)Lx * Ly * Lz, 256, 152 * 16), 256, 0, s>>>(out, comp, Lx, Ly, Lz, nx, ny, nz, h, k,
                                                                             sigma0, self);
  return cudaGetLastError();
}

cudaError_t launch_extract_octant(const double2* full, int Lx, int Ly, int Lz, double scale, double2* o64,
                                  float2* o32, void* odf, cudaStream_t s) {
  const long n = (long)(Lx / 2 + 1) * (Ly / 2 + 1) * (Lz / 2 + 1);
  k_extract_octant<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(full, Lx, Ly, Lz, scale, o64, o32,
                                                               reinterpret_cast<float4*>(odf));
  return cudaGetLastError();
}

cudaError_t launch_set_contrast(const double* s6, long N, double sigma0, double* d64, float* d32, int* bad,
                                cudaStream_t s) {
  k_set_contrast<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(s6, N, sigma0, d64, d32, bad);
  return cudaGetLastError();
}

cudaError_t launch_plane_active(const double* d64, long N, long nxy, int nz, int* act, cudaStream_t s) {
  k_plane_active<<<nz, 256, 0, s>>>(d64, N, nxy, act);
  return cudaGetLastError();
}
cudaError_t launch_contract_tensors(const double* d64, long N, double sigma0, double* K64, double* M64, float* K32,
                                    float* M32, cudaStream_t s) {
  k_contract_tensors<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(d64, N, sigma0, K64, M64, K32, M32);
  return cudaGetLastError();
}
cudaError_t launch_apply_sym6(const float* M, long m_cs, float2* x, long cs, long n, cudaStream_t s) {
  k_apply_sym6<float2, float><<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(M, m_cs, x, cs, n);
  return cudaGetLastError();
}
cudaError_t launch_apply_sym6(const double* M, long m_cs, double2* x, long cs, long n, cudaStream_t s) {
  k_apply_sym6<double2, double><<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(M, m_cs, x, cs, n);
  return cudaGetLastError();
}

cudaError_t launch_incident_E(double2* E0, int nx, int ny, int nz, const double* origin, double h, const double* pos,
                              const double* m, double2 k, double omega_mu0, cudaStream_t s) {
  const long N = (long)nx * ny * nz;
  k_incident_E<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(E0, nx, ny, nz, origin[0], origin[1], origin[2], h, pos[0],
                                                           pos[1], pos[2], m[0], m[1], m[2], k, omega_mu0);
  return cudaGetLastError();
}

int receivers_partials_blocks(long N) { return (int)grid_for(N, 256, 152 * 4); }

cudaError_t launch_receivers(const double2* E, long e_cs, const double* ds, long N, int nx, int ny, const double* origin,
                             double h, const double* rx_dev, int n_rx, double2 k, double2* part, const double* src_pos,
                             const double* m, double2* H, cudaStream_t s) {
  const int nblk = receivers_partials_blocks(N);
  k_receivers<<<nblk, 256, 0, s>>>(E, e_cs, ds, N, nx, ny, origin[0], origin[1], origin[2], h, rx_dev, n_rx, k, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_receivers_finish<<<1, 32 * ((n_rx * 3 + 31) / 32), 0, s>>>(part, nblk, rx_dev, n_rx, src_pos[0], src_pos[1],
                                                               src_pos[2], m[0], m[1], m[2], k, H);
  return cudaGetLastError();
}

}  // namespace ie
