// icp.cu -- the depth tracker's linearised point-to-plane system (Section
// 4.1) on sm_103a, and its C ABI.
//
// The tracker renders a point map V and a normal map N of the model from a
// reference pose (the raycast, Section 4.4), projects every point of a new
// depth image onto them with the current pose estimate and measures its
// distance from the tangent plane there. The pose update minimising the
// linearised sum of squared distances solves a 6x6 system whose terms
// (H = sum J J^T, g = sum J r, E = sum r^2, the inlier count) are reduced
// here; the 6x6 solve stays on the host, as in the report.
//
//   normals: one thread per pixel, the normalised cross product of the
//            point map's central differences;
//   reduce:  a pass over the pixels (rows by CTA), the 29 terms
//            accumulated per thread and summed per warp and CTA in FP32;
//            every CTA writes its partial sums and the last CTA to finish
//            adds them as double-floats, in a fixed order (the result does
//            not depend on scheduling).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>

#include "scene_impl.h"

namespace tsdf {
namespace {

constexpr int kIcpTerms = 29;
constexpr int kIcpThreads = 256;
constexpr int kIcpCtasPerSm = 4;  // at most (the parameter form fits four)
constexpr int kIcpPartialsPerLane = 20;
constexpr int kIcpMaxCtas = 32 * kIcpPartialsPerLane;  // the last CTA's lanes hold them all

struct IcpConst {
  float Ri[9], ti[3];  // current camera -> world: P = Ri p + ti
  float Mr[9], tr[3];  // world -> reference camera
  float fx, fy, cx, cy, inv_fx, inv_fy;
  float max_d2;        // squared distance threshold
  int width, height;
  long long pitch;     // depth row pitch in elements
};

__global__ void __launch_bounds__(256) normals_kernel(const float4* __restrict__ pts,
                                                      float4* __restrict__ nrm, int width,
                                                      int height) {
  const int n = width * height;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int u = i % width, v = i / width;
    float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (u > 0 && v > 0 && u < width - 1 && v < height - 1) {
      const float4 c = pts[i], l = pts[i - 1], r = pts[i + 1], t = pts[i - width],
                   b = pts[i + width];
      if (c.w == 1.0f && l.w == 1.0f && r.w == 1.0f && t.w == 1.0f && b.w == 1.0f) {
        const float dux = r.x - l.x, duy = r.y - l.y, duz = r.z - l.z;
        const float dvx = b.x - t.x, dvy = b.y - t.y, dvz = b.z - t.z;
        const float x = duy * dvz - duz * dvy, y = duz * dvx - dux * dvz, z = dux * dvy - duy * dvx;
        const float len2 = x * x + y * y + z * z;
        if (len2 > 0.0f) {
          const float inv = 1.0f / sqrtf(len2);
          out = make_float4(x * inv, y * inv, z * inv, 1.0f);
        }
      }
    }
    nrm[i] = out;
  }
}

// One level of the depth hierarchy: per 2x2 block the mean of its valid
// depths (summed in a fixed order, then divided), 0 where none is valid.
__global__ void __launch_bounds__(256) downsample_kernel(const float* __restrict__ depth,
                                                         long long pitch, int w2, int h2,
                                                         float* __restrict__ out) {
  const int n = w2 * h2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int u = i % w2, v = i / w2;
    const float* r0 = depth + (size_t)(2 * v) * pitch + 2 * u;
    const float* r1 = r0 + pitch;
    const float q[4] = {__ldg(r0), __ldg(r0 + 1), __ldg(r1), __ldg(r1 + 1)};
    float sum = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (q[k] > 0.0f && q[k] < INFINITY) {
        sum += q[k];
        ++cnt;
      }
    out[i] = cnt ? __fdiv_rn(sum, (float)cnt) : 0.0f;
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(~0u, x, o);
  return x;
}

// An unevaluated sum hi + lo of floats (about 48 bits): the sum over CTAs
// keeps its precision without the FP64 pipe, which GB300 runs at a small
// fraction of the FP32 rate. Knuth's two-sum adds exactly.
struct Df {
  float hi, lo;
};
__device__ __forceinline__ Df df_add(Df a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  return Df{s, a.lo + ((a.hi - (s - bb)) + (b - bb))};
}
__device__ __forceinline__ Df df_add(Df a, Df b) {
  Df r = df_add(a, b.hi);
  r.lo += b.lo;
  return r;
}
__device__ __forceinline__ Df warp_sum(Df x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const Df y{__shfl_xor_sync(~0u, x.hi, o), __shfl_xor_sync(~0u, x.lo, o)};
    x = df_add(x, y);
  }
  return x;
}

// DEV: the constants come from device memory (written by icp_prepare_kernel
// from a pose that lives on the device), else from the launch parameters.
template <bool DEV>
__global__ void __launch_bounds__(kIcpThreads) icp_reduce_kernel(
    IcpConst kv, const IcpConst* __restrict__ kp, const float* __restrict__ depth,
    const float4* __restrict__ pts, const float4* __restrict__ nrm, float* __restrict__ partial,
    unsigned* ticket, double* __restrict__ out) {
  __shared__ float s_part[kIcpThreads / 32][kIcpTerms];
  __shared__ bool s_last;
  const IcpConst k = DEV ? *kp : kv;
  float acc[kIcpTerms];
#pragma unroll
  for (int t = 0; t < kIcpTerms; ++t) acc[t] = 0.0f;
  // rows by CTA, columns by thread
  for (int v = blockIdx.x; v < k.height; v += gridDim.x)
  for (int u = threadIdx.x; u < k.width; u += blockDim.x) {
    const float d = __ldg(depth + (size_t)v * k.pitch + u);
    if (!(d > 0.0f) || !(d < INFINITY)) continue;
    // the pixel's point, in the current camera and in the world
    const float px = d * (((float)u - k.cx) * k.inv_fx), py = d * (((float)v - k.cy) * k.inv_fy);
    float P[3], q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      P[r] = fmaf(k.Ri[3 * r], px, fmaf(k.Ri[3 * r + 1], py, fmaf(k.Ri[3 * r + 2], d, k.ti[r])));
#pragma unroll
    for (int r = 0; r < 3; ++r)
      q[r] = fmaf(k.Mr[3 * r], P[0], fmaf(k.Mr[3 * r + 1], P[1], fmaf(k.Mr[3 * r + 2], P[2], k.tr[r])));
    if (!(q[2] > 0.0f)) continue;
    // nearest reference pixel
    const float x = k.fx * q[0] / q[2] + k.cx, y = k.fy * q[1] / q[2] + k.cy;
    if (!(x >= -0.5f && y >= -0.5f && x < (float)k.width - 0.5f && y < (float)k.height - 0.5f))
      continue;
    const int ix = min((int)floorf(x + 0.5f), k.width - 1);
    const int iy = min((int)floorf(y + 0.5f), k.height - 1);
    const float4 V = __ldg(pts + (size_t)iy * k.width + ix);
    const float4 N = __ldg(nrm + (size_t)iy * k.width + ix);
    if (V.w != 1.0f || N.w != 1.0f) continue;
    const float dx = P[0] - V.x, dy = P[1] - V.y, dz = P[2] - V.z;
    if (dx * dx + dy * dy + dz * dz > k.max_d2) continue;
    const float r = dx * N.x + dy * N.y + dz * N.z;
    const float J[6] = {P[1] * N.z - P[2] * N.y, P[2] * N.x - P[0] * N.z, P[0] * N.y - P[1] * N.x,
                        N.x, N.y, N.z};
    int t = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) {
        acc[t] = fmaf(J[a], J[b], acc[t]);
        ++t;
      }
#pragma unroll
    for (int a = 0; a < 6; ++a) acc[21 + a] = fmaf(J[a], r, acc[21 + a]);
    acc[27] = fmaf(r, r, acc[27]);
    acc[28] += 1.0f;
  }
  // within the CTA in FP32 (a fixed tree: warps, then warps in order); the
  // per-thread and per-CTA sums are short, their FP32 error stays near
  // 1e-6 of the summed magnitudes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kIcpTerms; ++t) {
    const float s = warp_sum(acc[t]);
    if (lane == 0) s_part[warp][t] = s;
  }
  __syncthreads();
  if (threadIdx.x < kIcpTerms) {
    float s = 0.0f;
    for (int w = 0; w < kIcpThreads / 32; ++w) s += s_part[w][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;  // term-major
  }
  // the last CTA to finish adds the partial sums: warp w takes terms w,
  // w + 8, ...; for a term every lane loads its (at most 20) CTAs' partials
  // at once and adds them as a double-float, and the warp combines the lanes
  // (a fixed order, whatever the scheduling)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int t = warp; t < kIcpTerms; t += kIcpThreads / 32) {
    const float* pt = partial + (size_t)t * gridDim.x;
    float x[kIcpPartialsPerLane];
#pragma unroll
    for (int j = 0; j < kIcpPartialsPerLane; ++j) {
      const unsigned b = lane + 32u * j;
      x[j] = b < gridDim.x ? __ldcg(pt + b) : 0.0f;
    }
    Df s{0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < kIcpPartialsPerLane; ++j) s = df_add(s, x[j]);
    s = warp_sum(s);
    if (lane == 0) out[t] = (double)s.hi + (double)s.lo;
  }
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next reduction
}

// status bits of a handle (tsdf_icp_status)
constexpr int kIcpStPose = 1;      // a device pose was not an invertible affine map
constexpr int kIcpStSkipped = 2;   // a solve found fewer than 6 inliers: pose kept
constexpr int kIcpStSingular = 4;  // a solve met a system that is not positive definite

// The reduction's constants from a pose in device memory (one thread): the
// inverse of its rotation part by the adjugate, in FP64, rounded to float.
// `base` carries the rest (reference pose, intrinsics, sizes).
__global__ void icp_prepare_kernel(const double* __restrict__ pose, IcpConst base, IcpConst* out,
                                   int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  IcpConst k = base;
  const double* M = pose;
  const double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9],
               kk = M[10];
  const double det = a * (e * kk - f * h) - b * (d * kk - f * g) + c * (d * h - e * g);
  if (!(fabs(det) > 1e-300) || M[12] != 0.0 || M[13] != 0.0 || M[14] != 0.0 || M[15] != 1.0) {
    atomicOr(status, kIcpStPose);
    k.max_d2 = -1.0f;  // rejects every pixel: the solve then keeps the pose
    *out = k;
    return;
  }
  const double Ri[9] = {(e * kk - f * h) / det, (c * h - b * kk) / det, (b * f - c * e) / det,
                        (f * g - d * kk) / det, (a * kk - c * g) / det, (c * d - a * f) / det,
                        (d * h - e * g) / det,  (b * g - a * h) / det,  (a * e - b * d) / det};
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) k.Ri[3 * r + q] = (float)Ri[3 * r + q];
    k.ti[r] = (float)(-(Ri[3 * r] * M[3] + Ri[3 * r + 1] * M[7] + Ri[3 * r + 2] * M[11]));
  }
  *out = k;
}

// One Gauss-Newton step on the device (one thread, FP64): H x = -g by
// Cholesky from the 29 terms; x = (w, t) is a small motion of the world
// points, P' = exp(w) P + t, so the camera-to-world map is premultiplied by
// it and the pose (world -> camera) becomes M [exp(w) | t]^-1.
__global__ void icp_solve_kernel(const double* __restrict__ sums, double* pose, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!(sums[28] >= 6.0)) {
    atomicOr(status, kIcpStSkipped);
    return;
  }
  double A[6][6], x[6];
  int t = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) A[i][j] = A[j][i] = sums[t++];
  // Cholesky A = L L^T (L in the lower triangle of A)
  for (int j = 0; j < 6; ++j) {
    double dg = A[j][j];
    for (int q = 0; q < j; ++q) dg -= A[j][q] * A[j][q];
    if (!(dg > 0.0)) {
      atomicOr(status, kIcpStSingular);
      return;
    }
    A[j][j] = sqrt(dg);
    for (int i = j + 1; i < 6; ++i) {
      double v = A[i][j];
      for (int q = 0; q < j; ++q) v -= A[i][q] * A[j][q];
      A[i][j] = v / A[j][j];
    }
  }
  for (int i = 0; i < 6; ++i) {  // L y = -g
    double v = -sums[21 + i];
    for (int q = 0; q < i; ++q) v -= A[i][q] * x[q];
    x[i] = v / A[i][i];
  }
  for (int i = 5; i >= 0; --i) {  // L^T x = y
    double v = x[i];
    for (int q = i + 1; q < 6; ++q) v -= A[q][i] * x[q];
    x[i] = v / A[i][i];
  }
  // R = exp(w) (Rodrigues)
  const double th = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (th > 0.0) {
    const double kx = x[0] / th, ky = x[1] / th, kz = x[2] / th;
    const double s = sin(th), c1 = 1.0 - cos(th);
    const double K[9] = {0, -kz, ky, kz, 0, -kx, -ky, kx, 0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double kk = 0.0;
        for (int q = 0; q < 3; ++q) kk += K[3 * i + q] * K[3 * q + j];
        R[3 * i + j] += s * K[3 * i + j] + c1 * kk;
      }
  }
  // [R | t]^-1 = [R^T | -R^T t]; pose <- pose [R^T | -R^T t]
  double Rt[9], ti[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rt[3 * i + j] = R[3 * j + i];
  for (int i = 0; i < 3; ++i) ti[i] = -(Rt[3 * i] * x[3] + Rt[3 * i + 1] * x[4] + Rt[3 * i + 2] * x[5]);
  double Mn[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      Mn[4 * i + j] = pose[4 * i] * Rt[j] + pose[4 * i + 1] * Rt[3 + j] + pose[4 * i + 2] * Rt[6 + j];
    Mn[4 * i + 3] = pose[4 * i] * ti[0] + pose[4 * i + 1] * ti[1] + pose[4 * i + 2] * ti[2] + pose[4 * i + 3];
  }
  for (int i = 0; i < 12; ++i) pose[i] = Mn[i];
}

}  // namespace
}  // namespace tsdf

using namespace tsdf;

struct tsdf_icp {
  cudaStream_t stream;
  int device;
  int sm_count;
  float* partial;    // grid x 29 per-CTA sums
  unsigned* ticket;
  IcpConst* kdev;    // constants for reductions whose pose lives on the device
  int* status;       // kIcpSt* bits
  int grid[2];       // reduce CTAs: constants as parameters / in device memory
  long long launches;
};

namespace {

// as many CTAs as fit on the GPU at once (at most kIcpMaxCtas)
template <bool DEV>
int icp_grid_for(int sm_count) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, icp_reduce_kernel<DEV>, kIcpThreads, 0) !=
          cudaSuccess || b < 1)
    b = 1;
  return std::min(sm_count * std::min(b, kIcpCtasPerSm), kIcpMaxCtas);
}

bool pose_affine(const double* M) {
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(M[i])) return false;
  return M[12] == 0.0 && M[13] == 0.0 && M[14] == 0.0 && M[15] == 1.0;
}

}  // namespace

int tsdf_icp_create(void* stream, tsdf_icp** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  tsdf_icp* h = (tsdf_icp*)calloc(1, sizeof(tsdf_icp));
  if (!h) return TSDF_ERR_OUT_OF_MEMORY;
  h->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) {
    h->grid[0] = icp_grid_for<false>(h->sm_count);
    h->grid[1] = icp_grid_for<true>(h->sm_count);
    e = cudaMalloc((void**)&h->partial, (size_t)kIcpMaxCtas * kIcpTerms * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->ticket, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->kdev, sizeof(IcpConst));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaFree(h->partial);
    cudaFree(h->ticket);
    cudaFree(h->kdev);
    cudaFree(h->status);
    free(h);
    return cuda_fail(e);
  }
  *out = h;
  return TSDF_OK;
}

int tsdf_icp_destroy(tsdf_icp* h) {
  if (!h) return TSDF_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  cudaFree(h->partial);
  cudaFree(h->ticket);
  cudaFree(h->kdev);
  cudaFree(h->status);
  free(h);
  return TSDF_OK;
}

int tsdf_icp_normals(tsdf_icp* h, const float* points, float* normals, int32_t width,
                     int32_t height) {
  if (!h || !points || !normals || width < 3 || height < 3 || width > (1 << 16) ||
      height > (1 << 16))
    return TSDF_ERR_INVALID_ARG;
  if (((uintptr_t)points & 15) || ((uintptr_t)normals & 15)) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(h->device));
  normals_kernel<<<h->sm_count * 8, 256, 0, h->stream>>>((const float4*)points, (float4*)normals,
                                                         width, height);
  TSDF_CUDA(cudaGetLastError());
  h->launches += 1;
  return TSDF_OK;
}

namespace {
// checks shared by the reductions; the constants that do not depend on the
// current pose (reference pose, intrinsics, sizes)
int icp_base(const float* depth, int64_t pitch_elems, const tsdf_intrinsics* intr,
             const double* ref_world_to_cam, const float* points, const float* normals,
             float max_dist, const double* sums, IcpConst* kc) {
  if (!depth || !points || !normals || !sums || !ref_world_to_cam) return TSDF_ERR_INVALID_ARG;
  int rc = validate_intr(intr);
  if (rc) return rc;
  if (pitch_elems < intr->width || !(max_dist > 0.0f) || !std::isfinite(max_dist))
    return TSDF_ERR_INVALID_ARG;
  if (((uintptr_t)points & 15) || ((uintptr_t)normals & 15) || ((uintptr_t)sums & 7))
    return TSDF_ERR_INVALID_ARG;
  if (!pose_affine(ref_world_to_cam)) return TSDF_ERR_INVALID_ARG;
  *kc = IcpConst{};
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) kc->Mr[3 * r + q] = (float)ref_world_to_cam[4 * r + q];
    kc->tr[r] = (float)ref_world_to_cam[4 * r + 3];
  }
  kc->fx = intr->fx;
  kc->fy = intr->fy;
  kc->cx = intr->cx;
  kc->cy = intr->cy;
  kc->inv_fx = (float)(1.0 / (double)intr->fx);
  kc->inv_fy = (float)(1.0 / (double)intr->fy);
  kc->max_d2 = max_dist * max_dist;
  kc->width = intr->width;
  kc->height = intr->height;
  kc->pitch = pitch_elems;
  return TSDF_OK;
}
}  // namespace

int tsdf_icp_level_intrinsics(const tsdf_intrinsics* intr, int32_t level, tsdf_intrinsics* out) {
  if (!intr || !out || level < 0 || level > 15) return TSDF_ERR_INVALID_ARG;
  const int rc = tsdf::validate_intr(intr);
  if (rc) return rc;
  tsdf_intrinsics in = *intr;
  for (int l = 0; l < level; ++l) {  // a coarse pixel is the centre of a 2x2 block
    in.fx *= 0.5f;
    in.fy *= 0.5f;
    in.cx = (in.cx - 0.5f) * 0.5f;
    in.cy = (in.cy - 0.5f) * 0.5f;
    in.width /= 2;
    in.height /= 2;
  }
  *out = in;
  return TSDF_OK;
}

int tsdf_icp_downsample(tsdf_icp* h, const float* depth, int64_t pitch_elems, int32_t width,
                        int32_t height, float* out) {
  if (!h || !depth || !out || width < 2 || height < 2 || width > (1 << 16) || height > (1 << 16) ||
      pitch_elems < width)
    return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(h->device));
  downsample_kernel<<<h->sm_count * 4, 256, 0, h->stream>>>(depth, pitch_elems, width / 2,
                                                            height / 2, out);
  TSDF_CUDA(cudaGetLastError());
  h->launches += 1;
  return TSDF_OK;
}

int tsdf_icp_reduce(tsdf_icp* h, const float* depth, int64_t pitch_elems,
                    const tsdf_intrinsics* intr, const double cur_world_to_cam[16],
                    const double ref_world_to_cam[16], const float* points, const float* normals,
                    float max_dist, double* sums) {
  if (!h || !cur_world_to_cam) return TSDF_ERR_INVALID_ARG;
  IcpConst kc;
  int rc = icp_base(depth, pitch_elems, intr, ref_world_to_cam, points, normals, max_dist, sums, &kc);
  if (rc) return rc;
  if (!pose_affine(cur_world_to_cam)) return TSDF_ERR_INVALID_ARG;
  const double* M = cur_world_to_cam;
  const double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], hh = M[9],
               k = M[10];
  const double det = a * (e * k - f * hh) - b * (d * k - f * g) + c * (d * hh - e * g);
  if (!(std::fabs(det) > 1e-300)) return TSDF_ERR_INVALID_ARG;
  const double Ri[9] = {(e * k - f * hh) / det, (c * hh - b * k) / det, (b * f - c * e) / det,
                        (f * g - d * k) / det,  (a * k - c * g) / det,  (c * d - a * f) / det,
                        (d * hh - e * g) / det, (b * g - a * hh) / det, (a * e - b * d) / det};
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) kc.Ri[3 * r + q] = (float)Ri[3 * r + q];
    kc.ti[r] = (float)(-(Ri[3 * r] * M[3] + Ri[3 * r + 1] * M[7] + Ri[3 * r + 2] * M[11]));
  }
  TSDF_CUDA(cudaSetDevice(h->device));
  icp_reduce_kernel<false><<<h->grid[0], kIcpThreads, 0, h->stream>>>(
      kc, nullptr, depth, (const float4*)points, (const float4*)normals, h->partial, h->ticket,
      sums);
  TSDF_CUDA(cudaGetLastError());
  h->launches += 1;
  return TSDF_OK;
}

int tsdf_icp_solve(tsdf_icp* h, const double* sums, double* pose) {
  if (!h || !sums || !pose || ((uintptr_t)sums & 7) || ((uintptr_t)pose & 7))
    return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(h->device));
  icp_solve_kernel<<<1, 32, 0, h->stream>>>(sums, pose, h->status);
  TSDF_CUDA(cudaGetLastError());
  h->launches += 1;
  return TSDF_OK;
}

int tsdf_icp_track(tsdf_icp* h, const float* depth, int64_t pitch_elems,
                   const tsdf_intrinsics* intr, double* pose, const double ref_world_to_cam[16],
                   const float* points, const float* normals, float max_dist, int32_t iterations,
                   double* sums) {
  if (!h || !pose || ((uintptr_t)pose & 7) || iterations < 1 || iterations > 1000)
    return TSDF_ERR_INVALID_ARG;
  IcpConst kc;
  int rc = icp_base(depth, pitch_elems, intr, ref_world_to_cam, points, normals, max_dist, sums, &kc);
  if (rc) return rc;
  TSDF_CUDA(cudaSetDevice(h->device));
  for (int it = 0; it < iterations; ++it) {
    icp_prepare_kernel<<<1, 32, 0, h->stream>>>(pose, kc, h->kdev, h->status);
    icp_reduce_kernel<true><<<h->grid[1], kIcpThreads, 0, h->stream>>>(
        kc, h->kdev, depth, (const float4*)points, (const float4*)normals, h->partial, h->ticket,
        sums);
    icp_solve_kernel<<<1, 32, 0, h->stream>>>(sums, pose, h->status);
  }
  TSDF_CUDA(cudaGetLastError());
  h->launches += 3LL * iterations;
  return TSDF_OK;
}

int tsdf_icp_status(tsdf_icp* h, int32_t* status) {
  if (!h || !status) return TSDF_ERR_INVALID_ARG;
  TSDF_CUDA(cudaSetDevice(h->device));
  int v = 0;
  TSDF_CUDA(cudaMemcpyAsync(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  TSDF_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  TSDF_CUDA(cudaStreamSynchronize(h->stream));
  *status = v;
  return TSDF_OK;
}

int tsdf_icp_kernel_launches(tsdf_icp* h, int64_t* n) {
  if (!h || !n) return TSDF_ERR_INVALID_ARG;
  *n = h->launches;
  return TSDF_OK;
}
