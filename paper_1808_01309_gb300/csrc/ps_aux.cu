// Auxiliary kernels: integrating-factor tables, FP64 reductions (energy,
// diagnostics, shell spectrum) and the forcing box gather.
#include "ps_passes.cuh"

namespace ps {

// exp(-nu |k_axis|^2 dt/2) per retained index of each axis, evaluated in FP64
// (the factor of a mode is the product of its three axis factors).
template <typename T>
__global__ void k_if_tables(const Geo g, double nu, double dt, T* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.cx + g.cy + g.cz;
  if (i >= n) return;
  double k;
  if (i < g.cx) {
    k = i * g.sx;
  } else if (i < g.cx + g.cy) {
    const int j = i - g.cx;
    k = (j <= g.Ky ? j : j - g.cy) * g.sy;
  } else {
    const int j = i - g.cx - g.cy;
    k = (j <= g.Kz ? j : j - g.cz) * g.sz;
  }
  tab[i] = T(exp(-nu * k * k * dt * 0.5));
}

template <typename T>
cudaError_t launch_if_tables(const Geo& g, double nu, double dt, void* tab, cudaStream_t s) {
  const int n = g.cx + g.cy + g.cz;
  k_if_tables<T><<<(n + 255) / 256, 256, 0, s>>>(g, nu, dt, static_cast<T*>(tab));
  return cudaGetLastError();
}

// Fixed-order sum of n partials (deterministic): one CTA.
__global__ void k_sum_partials(const double* __restrict__ part, int n, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) *out = t;
}

cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(part, n, out);
  return cudaGetLastError();
}

// Largest |p|, |q|, |r| of the nonzero retained forcing modes.
template <typename T>
__global__ void k_forcing_extent(const Geo g, const Spec f, int* ext) {
  using V = typename cplx<T>::type;
  const long long total = (long long)g.nz * g.ny * g.nh;
  const V* fp = static_cast<const V*>(f.p);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % g.nh);
    const int qi = (int)((i / g.nh) % g.ny);
    const int ri = (int)(i / ((long long)g.nh * g.ny));
    const int q = sidx(qi, g.ny), r = sidx(ri, g.nz);
    if (!kept(g, p, q, r)) continue;
    bool nz = false;
    for (int c = 0; c < 3; ++c) {
      const V v = fp[c * f.cs + (long long)ri * f.zs + (long long)qi * f.ys + p];
      nz |= (v.x != 0 || v.y != 0);
    }
    if (nz) {
      atomicMax(ext + 0, p);
      atomicMax(ext + 1, q < 0 ? -q : q);
      atomicMax(ext + 2, r < 0 ? -r : r);
    }
  }
}

template <typename T>
cudaError_t launch_forcing_extent(const Geo& g, Spec f, int* ext, cudaStream_t s) {
  k_forcing_extent<T><<<1024, 256, 0, s>>>(g, f, ext);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_forcing_gather(const Geo g, const Spec f, int Fx, int Fy, int Fz, typename cplx<T>::type* box) {
  using V = typename cplx<T>::type;
  const int nxb = Fx + 1, nyb = 2 * Fy + 1, nzb = 2 * Fz + 1;
  const int per = nxb * nyb * nzb;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * per) return;
  const int c = i / per, rem = i % per;
  const int p = rem % nxb, q = (rem / nxb) % nyb - Fy, r = rem / (nxb * nyb) - Fz;
  V v = czero<V>();
  if (p < ncols(g) && kept(g, g.kx0 + p, q, r)) {  // p: local column of a kx slab
    const V* fp = static_cast<const V*>(f.p);
    v = fp[c * f.cs + (long long)rowof(r, f.zwrap) * f.zs + (long long)rowof(q, f.ywrap) * f.ys + p];
  }
  box[i] = v;
}

template <typename T>
cudaError_t launch_forcing_gather(const Geo& g, Spec f, int Fx, int Fy, int Fz, void* box, cudaStream_t s) {
  const int n = 3 * (Fx + 1) * (2 * Fy + 1) * (2 * Fz + 1);
  k_forcing_gather<T><<<(n + 255) / 256, 256, 0, s>>>(g, f, Fx, Fy, Fz, static_cast<typename cplx<T>::type*>(box));
  return cudaGetLastError();
}

// Spectral diagnostics, one CTA per retained kz plane; row blk of `part`
// holds [E, Omega, H, max|k.u|, E_B, H_c, H_m, E_P, spectrum(0..nshells-1)] of
// that plane (the magnetic entries only for eq = 1 (MHD): B = components
// 3..5; the potential energy 1/2 w |theta|^2 only for eq = 2 (Boussinesq):
// theta = component 3).
template <typename T>
__global__ void k_diag_spectral(const Geo g, const Spec u, double* part, int nshells, int eq) {
  const int mhd = eq == 1;
  using V = typename cplx<T>::type;
  __shared__ double red[32];
  const int iz = blockIdx.x;
  const int r = iz <= g.Kz ? iz : iz - g.cz;
  const V* up = static_cast<const V*>(u.p);
  double* row = part + (long long)blockIdx.x * (DIAG_HEAD + nshells);
  double e = 0, om = 0, h = 0, md = 0, eb = 0, hc = 0, hm = 0, ep = 0;
  const int per = g.cy * g.cx;
  for (int i = threadIdx.x; i < per; i += blockDim.x) {
    const int iy = i / g.cx, p = i % g.cx;
    const int q = iy <= g.Ky ? iy : iy - g.cy;
    if (!kept(g, p, q, r)) continue;
    const V* pm = up + (long long)rowof(r, u.zwrap) * u.zs + (long long)rowof(q, u.ywrap) * u.ys + p;
    const V a0 = pm[0], a1 = pm[u.cs], a2 = pm[2 * u.cs];
    const double ux = a0.x, uxi = a0.y, uy = a1.x, uyi = a1.y, uz = a2.x, uzi = a2.y;
    const double kx = p * g.sx, ky = q * g.sy, kz = r * g.sz;
    const double w = (p == 0) ? 1.0 : 2.0;
    const double u2 = ux * ux + uxi * uxi + uy * uy + uyi * uyi + uz * uz + uzi * uzi;
    // c = k x u (complex); omega = i c
    const double cxr = ky * uz - kz * uy, cxi = ky * uzi - kz * uyi;
    const double cyr = kz * ux - kx * uz, cyi = kz * uxi - kx * uzi;
    const double czr = kx * uy - ky * ux, czi = kx * uyi - ky * uxi;
    const double o2 = cxr * cxr + cxi * cxi + cyr * cyr + cyi * cyi + czr * czr + czi * czi;
    // Re(conj(a) i b) = -a.x b.y + a.y b.x, summed over components
    const double hel = -(ux * cxi) + uxi * cxr - (uy * cyi) + uyi * cyr - (uz * czi) + uzi * czr;
    const double dr = kx * ux + ky * uy + kz * uz, di = kx * uxi + ky * uyi + kz * uzi;
    e += 0.5 * w * u2;
    om += 0.5 * w * o2;
    h += w * hel;
    md = fmax(md, sqrt(dr * dr + di * di));
    if (mhd) {
      const V b0 = pm[3 * u.cs], b1 = pm[4 * u.cs], b2 = pm[5 * u.cs];
      const double bx = b0.x, bxi = b0.y, by = b1.x, byi = b1.y, bz = b2.x, bzi = b2.y;
      eb += 0.5 * w * (bx * bx + bxi * bxi + by * by + byi * byi + bz * bz + bzi * bzi);
      hc += w * (ux * bx + uxi * bxi + uy * by + uyi * byi + uz * bz + uzi * bzi);
      const double k2 = kx * kx + ky * ky + kz * kz;
      if (k2 > 0) {
        // A = i d/|k|^2 with d = k x B; Re(conj(i d) . B) = d.re . B.im - d.im . B.re
        const double dxr = ky * bz - kz * by, dxi = ky * bzi - kz * byi;
        const double dyr = kz * bx - kx * bz, dyi = kz * bxi - kx * bzi;
        const double dzr = kx * by - ky * bx, dzi = kx * byi - ky * bxi;
        const double re = (dxr * bxi - dxi * bx) + (dyr * byi - dyi * by) + (dzr * bzi - dzi * bz);
        hm += w * re / k2;
      }
    }
    if (eq == 2) {
      const V t = pm[3 * u.cs];
      ep += 0.5 * w * ((double)t.x * t.x + (double)t.y * t.y);
    }
    const int sh = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
    if (sh < nshells) atomicAdd(row + DIAG_HEAD + sh, 0.5 * w * u2);
  }
  const double te = block_sum(e, red);
  const double to = block_sum(om, red);
  const double th = block_sum(h, red);
  const double tm = block_max(md, red);
  const double teb = block_sum(eb, red);
  const double thc = block_sum(hc, red);
  const double thm = block_sum(hm, red);
  const double tep = block_sum(ep, red);
  if (threadIdx.x == 0) {
    row[0] = te;
    row[1] = to;
    row[2] = th;
    row[3] = tm;
    row[4] = teb;
    row[5] = thc;
    row[6] = thm;
    row[7] = tep;
  }
}

template <typename T>
cudaError_t launch_diag_spectral(const Geo& g, Spec u, double* part, int nshells, int eq, cudaStream_t s) {
  k_diag_spectral<T><<<g.cz, 256, 0, s>>>(g, u, part, nshells, eq);
  return cudaGetLastError();
}

__global__ void k_diag_final(const double* __restrict__ part, int nblk, int nshells, double* out) {
  const int w = DIAG_HEAD + nshells;
  for (int j = threadIdx.x; j < w; j += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const double x = part[(long long)b * w + j];
      v = (j == 3) ? fmax(v, x) : v + x;
    }
    out[j] = v;
  }
}

cudaError_t launch_diag_final(const double* part, int nblk, int nshells, double* out, cudaStream_t s) {
  k_diag_final<<<1, 256, 0, s>>>(part, nblk, nshells, out);
  return cudaGetLastError();
}

// Contiguous copy of n bytes by the SMs (16-byte accesses, four in flight
// per thread); either side may be page-locked host memory addressed through
// its device mapping.
__global__ void k_stream_copy(const uint4* __restrict__ src, uint4* __restrict__ dst, long long n16) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

__global__ void k_stream_copy8(const uint2* __restrict__ src, uint2* __restrict__ dst, long long n8) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_stream_copy(const void* src, void* dst, size_t bytes, int nsm, cudaStream_t s) {
  const int blocks = 4 * (nsm > 0 ? nsm : 152);
  if (((uintptr_t)src | (uintptr_t)dst | bytes) % 16 == 0)
    k_stream_copy<<<blocks, 256, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst),
                                        (long long)(bytes / 16));
  else
    k_stream_copy8<<<blocks, 256, 0, s>>>(static_cast<const uint2*>(src), static_cast<uint2*>(dst),
                                         (long long)(bytes / 8));
  return cudaGetLastError();
}

// Copy the modes of the retained cube |p| <= Kx, |q| <= Ky, |r| <= Kz of nc
// caller-layout components from src to dst (either may be the device mapping
// of page-locked host memory); one kx row segment per group of threads.
template <typename V>
__global__ void k_copy_cube(const V* __restrict__ src, V* __restrict__ dst, const Geo g, int nc) {
  const long long rows = (long long)nc * g.cz * g.cy;
  const long long fcs = (long long)g.nz * g.ny * g.nh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows * g.cx;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % g.cx);
    const long long row = i / g.cx;
    const int iy = (int)(row % g.cy), iz = (int)((row / g.cy) % g.cz), c = (int)(row / ((long long)g.cy * g.cz));
    const int q = iy <= g.Ky ? iy : iy - g.cy, r = iz <= g.Kz ? iz : iz - g.cz;
    const long long o = c * fcs + ((long long)rowof(r, g.nz) * g.ny + rowof(q, g.ny)) * g.nh + p;
    dst[o] = src[o];
  }
}

cudaError_t launch_copy_cube(const void* src, void* dst, const Geo& g, int nc, size_t vb, int nsm, cudaStream_t s) {
  const int blocks = 8 * (nsm > 0 ? nsm : 152);
  if (vb == 8)
    k_copy_cube<float2><<<blocks, 256, 0, s>>>(static_cast<const float2*>(src), static_cast<float2*>(dst), g, nc);
  else
    k_copy_cube<double2><<<blocks, 256, 0, s>>>(static_cast<const double2*>(src), static_cast<double2*>(dst), g, nc);
  return cudaGetLastError();
}

template cudaError_t launch_if_tables<float>(const Geo&, double, double, void*, cudaStream_t);
template cudaError_t launch_if_tables<double>(const Geo&, double, double, void*, cudaStream_t);
template cudaError_t launch_forcing_extent<float>(const Geo&, Spec, int*, cudaStream_t);
template cudaError_t launch_forcing_extent<double>(const Geo&, Spec, int*, cudaStream_t);
template cudaError_t launch_forcing_gather<float>(const Geo&, Spec, int, int, int, void*, cudaStream_t);
template cudaError_t launch_forcing_gather<double>(const Geo&, Spec, int, int, int, void*, cudaStream_t);
template cudaError_t launch_diag_spectral<float>(const Geo&, Spec, double*, int, int, cudaStream_t);
template cudaError_t launch_diag_spectral<double>(const Geo&, Spec, double*, int, int, cudaStream_t);

}  // namespace ps
