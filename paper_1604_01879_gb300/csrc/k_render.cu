// Projection front end (Sec. 2.1): scale and translation normalisation of
// every mesh, then N_v = n_az * n_el depth-buffer views from cameras on the
// unit sphere, each looking at the origin.
//
// Normalisation: the area-weighted centroid of the surface goes to the origin
// (two-float FP32 sums, one block per mesh) and the largest vertex distance
// from it becomes 1. Views: orthographic along the camera's forward axis f, image axes
// r = f x z / |f x z| and u = r x f, the image spanning [-1, 1]^2 (the unit
// sphere's silhouette); depth = p . f + 1 in [0, 2], 2 where nothing is seen.
// One thread per (triangle, view) projects the triangle, walks the pixel
// centres of its bounding box, keeps those with all three edge functions >= 0
// (orientation made positive; degenerate triangles cover nothing) and writes
// the interpolated depth with atomicMin on the float bits (non-negative floats
// order like their bit patterns).
#include <cmath>

#include "gift_internal.cuh"

namespace gift {

namespace {

constexpr int kRenderT = 256;

__device__ __forceinline__ int find_mesh(const int64_t* __restrict__ off, int M, int64_t t) {
  int lo = 0, hi = M;  // off[lo] <= t < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// per mesh: (cx, cy, cz) = sum(area * centroid) / sum(area); per-triangle terms
// in FP32, sums in two-float arithmetic (no FP64 on the GPU)
__global__ __launch_bounds__(kRenderT) void k_mesh_centre(const float* __restrict__ V, const int32_t* __restrict__ T,
                                                          const int64_t* __restrict__ voff,
                                                          const int64_t* __restrict__ toff, float* __restrict__ centre) {
  const int m = blockIdx.x;
  const float* Vm = V + voff[m] * 3;
  F2 acc[4];
  for (int64_t t = toff[m] + threadIdx.x; t < toff[m + 1]; t += blockDim.x) {
    const int32_t* tr = T + t * 3;
    float a[3], b[3], c[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = Vm[(int64_t)tr[0] * 3 + d];
      b[d] = Vm[(int64_t)tr[1] * 3 + d];
      c[d] = Vm[(int64_t)tr[2] * 3 + d];
    }
    const float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const float e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const float cx = e1[1] * e2[2] - e1[2] * e2[1];
    const float cy = e1[2] * e2[0] - e1[0] * e2[2];
    const float cz = e1[0] * e2[1] - e1[1] * e2[0];
    const float area = 0.5f * sqrtf(cx * cx + cy * cy + cz * cz);
    for (int d = 0; d < 3; ++d) f2_add(acc[d], area * ((a[d] + b[d] + c[d]) * (1.f / 3.f)));
    f2_add(acc[3], area);
  }
  __shared__ F2 red[4][kRenderT / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 4; ++k) {
    F2 x = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = f2_merge(x, f2_shfl_xor(x, o));
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    F2 tot[4];
    for (int k = 0; k < 4; ++k)
      for (int i = 0; i < kRenderT / 32; ++i) tot[k] = f2_merge(tot[k], red[k][i]);
    const float A = f2_value(tot[3]);
    for (int d = 0; d < 3; ++d) centre[m * 4 + d] = A > 0.f ? __fdiv_rn(f2_value(tot[d]), A) : 0.f;
  }
}

// per mesh: scale = 1 / max_v |v - centre|
__global__ __launch_bounds__(kRenderT) void k_mesh_scale(const float* __restrict__ V, const int64_t* __restrict__ voff,
                                                         float* __restrict__ centre) {
  const int m = blockIdx.x;
  const float c0 = centre[m * 4], c1 = centre[m * 4 + 1], c2 = centre[m * 4 + 2];
  float mx = 0.f;
  for (int64_t v = voff[m] + threadIdx.x; v < voff[m + 1]; v += blockDim.x) {
    const float dx = V[v * 3] - c0, dy = V[v * 3 + 1] - c1, dz = V[v * 3 + 2] - c2;
    mx = fmaxf(mx, dx * dx + dy * dy + dz * dz);
  }
  __shared__ float red[kRenderT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int i = 0; i < kRenderT / 32; ++i) r = fmaxf(r, red[i]);
    centre[m * 4 + 3] = r > 0.f ? 1.f / sqrtf(r) : 1.f;
  }
}

// every vertex index must address its own mesh's vertices
__global__ void k_check_tris(const int32_t* __restrict__ T, const int64_t* __restrict__ voff,
                             const int64_t* __restrict__ toff, int M, int* __restrict__ bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= toff[M]) return;
  const int m = find_mesh(toff, M, t);
  const int64_t nv = voff[m + 1] - voff[m];
  for (int k = 0; k < 3; ++k) {
    const int32_t i = T[t * 3 + k];
    if (i < 0 || i >= nv) atomicExch(bad, 1);
  }
}

__global__ void k_fill_depth(float* __restrict__ p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 2.f;
}

// thread per (triangle, view); frames [Nv, 9] = (r, u, f)
__global__ __launch_bounds__(kRenderT) void k_render(const float* __restrict__ V, const int32_t* __restrict__ T,
                                                     const int64_t* __restrict__ voff,
                                                     const int64_t* __restrict__ toff, int M,
                                                     const float* __restrict__ cs, const float* __restrict__ frames,
                                                     int Nv, int H, int W, float* __restrict__ depth) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = toff[M] * Nv;
  if (idx >= total) return;
  const int v = (int)(idx % Nv);
  const int64_t t = idx / Nv;
  const int m = find_mesh(toff, M, t);
  const float* fr = frames + v * 9;
  const float c0 = cs[m * 4], c1 = cs[m * 4 + 1], c2 = cs[m * 4 + 2], sc = cs[m * 4 + 3];
  float sx[3], sy[3], sz[3];
  for (int k = 0; k < 3; ++k) {
    const int64_t vi = voff[m] + T[t * 3 + k];
    const float px = (V[vi * 3] - c0) * sc, py = (V[vi * 3 + 1] - c1) * sc, pz = (V[vi * 3 + 2] - c2) * sc;
    sx[k] = px * fr[0] + py * fr[1] + pz * fr[2];
    sy[k] = px * fr[3] + py * fr[4] + pz * fr[5];
    sz[k] = px * fr[6] + py * fr[7] + pz * fr[8] + 1.f;
  }
  float area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sy[1] - sy[0]) * (sx[2] - sx[0]);
  if (area == 0.f) return;
  if (area < 0.f) {  // orient to a positive area
    float tx = sx[1], ty = sy[1], tz = sz[1];
    sx[1] = sx[2]; sy[1] = sy[2]; sz[1] = sz[2];
    sx[2] = tx; sy[2] = ty; sz[2] = tz;
    area = -area;
  }
  const float xmin = fminf(sx[0], fminf(sx[1], sx[2])), xmax = fmaxf(sx[0], fmaxf(sx[1], sx[2]));
  const float ymin = fminf(sy[0], fminf(sy[1], sy[2])), ymax = fmaxf(sy[0], fmaxf(sy[1], sy[2]));
  // pixel centres x_j = -1 + (2j + 1) / W, y_i = 1 - (2i + 1) / H inside the box
  const int j0 = max(0, (int)ceilf((xmin + 1.f) * 0.5f * W - 0.5f) - 1);
  const int j1 = min(W - 1, (int)floorf((xmax + 1.f) * 0.5f * W - 0.5f) + 1);
  const int i0 = max(0, (int)ceilf((1.f - ymax) * 0.5f * H - 0.5f) - 1);
  const int i1 = min(H - 1, (int)floorf((1.f - ymin) * 0.5f * H - 0.5f) + 1);
  float* img = depth + ((int64_t)m * Nv + v) * H * W;
  const float inv_area = 1.f / area;
  for (int i = i0; i <= i1; ++i) {
    const float py = 1.f - (float)(2 * i + 1) / (float)H;
    if (py < ymin || py > ymax) continue;
    for (int j = j0; j <= j1; ++j) {
      const float px = -1.f + (float)(2 * j + 1) / (float)W;
      if (px < xmin || px > xmax) continue;
      const float ea = (sx[2] - sx[1]) * (py - sy[1]) - (sy[2] - sy[1]) * (px - sx[1]);
      const float eb = (sx[0] - sx[2]) * (py - sy[2]) - (sy[0] - sy[2]) * (px - sx[2]);
      const float ec = (sx[1] - sx[0]) * (py - sy[0]) - (sy[1] - sy[0]) * (px - sx[0]);
      if (ea < 0.f || eb < 0.f || ec < 0.f) continue;
      const float z = fminf(fmaxf((ea * sz[0] + eb * sz[1] + ec * sz[2]) * inv_area, 0.f), 2.f);
      atomicMin(reinterpret_cast<int*>(img + (int64_t)i * W + j), __float_as_int(z));
    }
  }
}

}  // namespace

void render_views(const float* V, const int32_t* T, const std::vector<int64_t>& h_voff,
                  const std::vector<int64_t>& h_toff, int M, int n_az, int n_el, int H, int W, float* depth,
                  Scratch& sc, cudaStream_t s) {
  const int Nv = n_az * n_el;
  // camera frames in float64 on the host: r, u, f per view (view = el_index * n_az + az_index)
  std::vector<float> fr((size_t)Nv * 9);
  for (int je = 0; je < n_el; ++je)
    for (int ia = 0; ia < n_az; ++ia) {
      const double az = 2.0 * M_PI * ia / n_az;
      const double el = M_PI * ((je + 0.5) / n_el - 0.5);
      const double f[3] = {-cos(el) * cos(az), -cos(el) * sin(az), -sin(el)};
      double r[3] = {f[1], -f[0], 0.0};  // f x (0, 0, 1)
      const double rn = sqrt(r[0] * r[0] + r[1] * r[1]);
      r[0] /= rn;
      r[1] /= rn;
      const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
      float* o = fr.data() + (size_t)(je * n_az + ia) * 9;
      for (int d = 0; d < 3; ++d) {
        o[d] = (float)r[d];
        o[3 + d] = (float)u[d];
        o[6 + d] = (float)f[d];
      }
    }
  float* d_fr = sc.get<float>(fr.size());
  GIFT_CUDA(cudaMemcpyAsync(d_fr, fr.data(), fr.size() * 4, cudaMemcpyHostToDevice, s));
  int64_t* voff = sc.get<int64_t>((size_t)M + 1);
  int64_t* toff = sc.get<int64_t>((size_t)M + 1);
  GIFT_CUDA(cudaMemcpyAsync(voff, h_voff.data(), ((size_t)M + 1) * 8, cudaMemcpyHostToDevice, s));
  GIFT_CUDA(cudaMemcpyAsync(toff, h_toff.data(), ((size_t)M + 1) * 8, cudaMemcpyHostToDevice, s));
  if (h_toff[M] > 0) {
    int* bad = sc.get<int>(1);
    GIFT_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_check_tris<<<(unsigned)cdiv(h_toff[M], 256), 256, 0, s>>>(T, voff, toff, M, bad);
    GIFT_LAUNCHED("k_check_tris");
    int h_bad = 0;
    GIFT_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    GIFT_CUDA(cudaStreamSynchronize(s));
    if (h_bad) fail(GIFT_EINVAL, "a triangle addresses a vertex outside its mesh");
  }
  float* cs = sc.get<float>((size_t)M * 4);
  k_mesh_centre<<<(unsigned)M, kRenderT, 0, s>>>(V, T, voff, toff, cs);
  GIFT_LAUNCHED("k_mesh_centre");
  k_mesh_scale<<<(unsigned)M, kRenderT, 0, s>>>(V, voff, cs);
  GIFT_LAUNCHED("k_mesh_scale");
  const int64_t npix = (int64_t)M * Nv * H * W;
  k_fill_depth<<<(unsigned)cdiv(npix, 256), 256, 0, s>>>(depth, npix);
  GIFT_LAUNCHED("k_fill_depth");
  const int64_t work = h_toff[M] * Nv;
  if (work > 0) {
    k_render<<<(unsigned)cdiv(work, kRenderT), kRenderT, 0, s>>>(V, T, voff, toff, M, cs, d_fr, Nv, H, W, depth);
    GIFT_LAUNCHED("k_render");
  }
}

}  // namespace gift
