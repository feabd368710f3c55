// stream3d.cu -- one X-MCGS sweep (both colour phases) of a 3D float32 level in one pass over memory.
//
// A sweep updates the cells of the first colour from the old values of the second (phase 1), then the
// cells of the second colour from the new values of the first (phase 2; Sec. 2.3, Eqs. FCGS-1..4 and
// the 3D sets of Appendix B, read as red-black phases). Phase 1 at plane p needs the old planes p-1
// and p+1; phase 2 at plane p needs phase 1 done at planes p-1, p and p+1. A block therefore walks a
// segment of planes z and, at step t, runs phase 1 at plane t+1 and phase 2 at plane t-1: the
// two phases stream through memory one after the other, two planes apart, and each plane of u and f
// is read once and written once per sweep (the two colour launches of the per-operation path read
// and write it twice, and re-read neighbouring planes).
//
// Layout of the work: a block of R+2 warps owns a 128-column strip of R consecutive rows y; warp w
// handles row y0-1+w, lane L the four cells x0 = xs + 4L .. x0+3 (float4). The rows y0-1 and y0+R
// (warps 0 and R+1) and the columns xs-1 and xs+128 (lanes 0 and 31) are halos: phase 1 is computed
// there too, because phase 2 at the strip's edge reads it, but only the R x 128 interior is written.
// The planes arrive in shared memory as TMA tiles two steps ahead of their use -- old u over rows
// y0-2 .. y0+R+1 and columns xs-4 .. xs+131 (out-of-range cells read as zero), f over rows
// y0-1 .. y0+R -- in rings of slots whose mbarriers the copies complete; every wait is bounded (the
// kernel then sets an error word the host reports as FAS_ETIMEOUT). Phase 1 writes its values to a
// ring of plane buffers that phase 2 reads. One barrier per step. Because blocks recompute each
// other's halos, u is read from one buffer and written to another.
//
// Arithmetic per point is point_update's expression (same association and fma placement), so the
// sweep equals the two colour launches of k_smooth_colour4 bit for bit.
#include <algorithm>

#include "common.cuh"
#include "stream3d.h"
#include "tma.cuh"

namespace fasmg {
namespace {

constexpr int kS3Rows = 14;                // interior rows per block
constexpr int kS3Warps = kS3Rows + 2;      // + the two halo rows
constexpr int kS3Threads = 32 * kS3Warps;  // 512
constexpr int kS3Cols = 128;               // strip width
constexpr int kS3Pitch = kS3Cols + 8;      // tile row: x = xs-4 .. xs+131
constexpr int kS3Off = 4;                  // tile column of x = xs
constexpr int kUTileRows = kS3Rows + 4;    // old u: rows y0-2 .. y0+R+1
constexpr int kFTileRows = kS3Rows + 2;    // f and phase-1 values: rows y0-1 .. y0+R
constexpr int kUSlot = 2464;               // floats per u slot (kS3Pitch * kUTileRows = 2448, padded to 128 bytes)
constexpr int kFSlot = kS3Pitch * kFTileRows;  // 2176 floats (8704 bytes, a multiple of 128)
constexpr int kUDepth = 4, kFDepth = 4, kNDepth = 4;
constexpr int kNBar3 = kUDepth + kFDepth;
constexpr size_t kS3Smem = (size_t)(kUDepth * kUSlot + (kFDepth + kNDepth) * kFSlot) * sizeof(float) +
                           kNBar3 * sizeof(uint64_t) + 128;

__device__ __forceinline__ int mod(int a, int m) { return ((a % m) + m) % m; }

__device__ __forceinline__ float4 ld4s(const float* row, int lane) {
  return reinterpret_cast<const float4*>(row + kS3Off)[lane];
}

__device__ __forceinline__ float& comp(float4& q, int k) { return k == 0 ? q.x : (k == 1 ? q.y : (k == 2 ? q.z : q.w)); }
__device__ __forceinline__ float compc(const float4& q, int k) { return k == 0 ? q.x : (k == 1 ? q.y : (k == 2 ? q.z : q.w)); }
__device__ __forceinline__ float4 phase4(const float* row, const float* rs, const float* rn, const float4& bo,
                                         const float4& to, const float4& fv, const LevelDesc<float>& L, int x0, int y,
                                         int z, int c, int lane) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const float4 old = ld4s(row, lane);
  const float4 sv = ld4s(rs, lane);
  const float4 nv = ld4s(rn, lane);
  const float wl = row[kS3Off + 4 * lane - 1], er = row[kS3Off + 4 * lane + 4];
  float4 cur = old;
  const int k0 = (x0 + y + z + 3 + c) & 1;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = k0 + 2 * kk;
    const int x = x0 + k;
    const float w = x > 0 ? (k > 0 ? compc(old, k - 1) : wl) : 0.f;
    const float e = x < nx - 1 ? (k < 3 ? compc(old, k + 1) : er) : 0.f;
    const float s = y > 0 ? compc(sv, k) : 0.f;
    const float n = y < ny - 1 ? compc(nv, k) : 0.f;
    float acc = (w + e) + (s + n);
    const float b = z > 0 ? compc(bo, k) : 0.f;
    const float t = z < nz - 1 ? compc(to, k) : 0.f;
    acc = acc + (b + t);
    const int cls = bclass<3>(x, y, z, nx, ny, nz);
    comp(cur, k) = fmaf(L.a[cls], acc, L.b[cls] * compc(fv, k));
  }
  return cur;
}

// Phase 1 at a halo column cell (x, y, z) of tile column col (old values); returns its value after
// phase 1 (the old one when it has the other colour).
__device__ __forceinline__ float phase1_halo(const float* row, const float* rs, const float* rn, int col, float bo,
                                             float to, float fv, const LevelDesc<float>& L, int x, int y, int z,
                                             int c) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const float old = row[col];
  if (x < 0 || x >= nx || ((x + y + z + 3 + c) & 1)) return old;
  const float w = x > 0 ? row[col - 1] : 0.f;
  const float e = x < nx - 1 ? row[col + 1] : 0.f;
  const float s = y > 0 ? rs[col] : 0.f;
  const float n = y < ny - 1 ? rn[col] : 0.f;
  float acc = (w + e) + (s + n);
  const float b = z > 0 ? bo : 0.f;
  const float t = z < nz - 1 ? to : 0.f;
  acc = acc + (b + t);
  const int cls = bclass<3>(x, y, z, nx, ny, nz);
  return fmaf(L.a[cls], acc, L.b[cls] * fv);
}

__global__ void __launch_bounds__(kS3Threads, 2)
    k_sweep3d(float* __restrict__ uout, const __grid_constant__ CUtensorMap tu, const __grid_constant__ CUtensorMap tf,
              LevelDesc<float> L, int c1, int zseg, unsigned* err, unsigned long long wait_ns, int withhold) {
  extern __shared__ __align__(128) unsigned char smem_s3[];
  float* su = reinterpret_cast<float*>(smem_s3 + ((128u - (smem_u32(smem_s3) & 127u)) & 127u));
  float* sf = su + kUDepth * kUSlot;
  float* sn = sf + kFDepth * kFSlot;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sn + kNDepth * kFSlot);  // u slots, then f slots
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int c2 = 1 - c1;
  const int nstrips = nx / kS3Cols;
  const int nyg = (ny + kS3Rows - 1) / kS3Rows;
  const int nzs = (nz + zseg - 1) / zseg;
  const int ntasks = nstrips * nyg * nzs;
  if (tid == 0) {
    for (int k = 0; k < kNBar3; ++k) mbar_init(bar + k, 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t par = 0u, pend = 0u;
  bool aborted = false;
  auto wait_bar = [&](int k) -> bool {
    const bool ok = mbar_wait_bounded(bar + k, (par >> k) & 1u, wait_ns);
    par ^= 1u << k;
    if (tid == 0 && ok) pend &= ~(1u << k);
    return ok;
  };
  for (int task = blockIdx.x; task < ntasks && !aborted; task += gridDim.x) {
    const int xs = (task % nstrips) * kS3Cols;
    const int rest = task / nstrips;
    const int y0 = (rest % nyg) * kS3Rows;
    const int z0 = (rest / nyg) * zseg, z1 = min(nz, z0 + zseg);
    const int y = y0 - 1 + w;
    const int x0 = xs + 4 * lane;
    const bool row_in = y >= 0 && y < ny;
    const bool interior = w >= 1 && w <= kS3Rows && row_in;
    auto u_ok = [&](int z) { return z >= 0 && z < nz && z >= z0 - 2 && z <= z1 + 1; };
    auto f_ok = [&](int z) { return z >= 0 && z < nz && z >= z0 - 1 && z <= z1; };
    auto issue_u = [&](int z) {
      const int k = mod(z, kUDepth);
      mbar_expect_tx(bar + k, kS3Pitch * kUTileRows * (uint32_t)sizeof(float));
      tma_load_3d(su + k * kUSlot, &tu, xs - kS3Off, y0 - 2, z, bar + k);
      pend |= 1u << k;
    };
    auto issue_f = [&](int z) {
      const int k = kUDepth + mod(z, kFDepth);
      mbar_expect_tx(bar + k, kFSlot * (uint32_t)sizeof(float));
      tma_load_3d(sf + mod(z, kFDepth) * kFSlot, &tf, xs - kS3Off, y0 - 1, z, bar + k);
      pend |= 1u << k;
    };
    // the test hook withholds one copy (block 0, first task): its waits must run out
    const bool hold = withhold && blockIdx.x == 0 && task == (int)blockIdx.x;
    if (tid == 0) {
      fence_async_smem();  // the previous task's reads of the slots come before the new copies
      for (int z = z0 - 2; z <= z0; ++z)
        if (u_ok(z) && !(hold && z == z0)) issue_u(z);
      if (f_ok(z0 - 1)) issue_f(z0 - 1);
    }
    bool ok = true;
    for (int z = z0 - 2; z <= z0 - 1; ++z)
      if (u_ok(z)) ok = wait_bar(mod(z, kUDepth)) && ok;
    for (int t = z0 - 2; t <= z1; ++t) {
      if (u_ok(t + 2)) ok = wait_bar(mod(t + 2, kUDepth)) && ok;
      if (f_ok(t + 1)) ok = wait_bar(kUDepth + mod(t + 1, kFDepth)) && ok;
      // the planes this step reads are in place; the slots it refills were last read two steps ago
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0) {
        fence_async_smem();
        if (u_ok(t + 3)) issue_u(t + 3);  // into the slot of plane t-1
        if (f_ok(t + 2)) issue_f(t + 2);  // into the slot of plane t-2
      }
      // phase 1 at plane p = t+1, from the old planes p-1, p, p+1
      const int p = t + 1;
      if (p <= z1 && p >= 0 && p < nz && row_in) {
        const float* U0 = su + mod(p, kUDepth) * kUSlot;
        const float* Ub = su + mod(p - 1, kUDepth) * kUSlot + (w + 1) * kS3Pitch;
        const float* Ut = su + mod(p + 1, kUDepth) * kUSlot + (w + 1) * kS3Pitch;
        const float* F = sf + mod(p, kFDepth) * kFSlot + w * kS3Pitch;
        const float* row = U0 + (w + 1) * kS3Pitch;
        const float4 v = phase4(row, row - kS3Pitch, row + kS3Pitch, ld4s(Ub, lane), ld4s(Ut, lane), ld4s(F, lane), L,
                                x0, y, p, c1, lane);
        float* nrow = sn + mod(p, kNDepth) * kFSlot + w * kS3Pitch;
        reinterpret_cast<float4*>(nrow + kS3Off)[lane] = v;
        if (lane == 0 || lane == 31) {
          const int col = lane == 0 ? kS3Off - 1 : kS3Off + kS3Cols;
          const int xh = lane == 0 ? xs - 1 : xs + kS3Cols;
          nrow[col] = phase1_halo(row, row - kS3Pitch, row + kS3Pitch, col, Ub[col], Ut[col], F[col], L, xh, y, p, c1);
        }
      }
      // phase 2 at plane q = t-1, from the phase-1 values of the planes q-1, q, q+1
      const int q = t - 1;
      if (q >= z0 && q < z1 && interior) {
        const float* row = sn + mod(q, kNDepth) * kFSlot + w * kS3Pitch;
        const float* Nb = sn + mod(q - 1, kNDepth) * kFSlot + w * kS3Pitch;
        const float* Nt = sn + mod(q + 1, kNDepth) * kFSlot + w * kS3Pitch;
        const float* F = sf + mod(q, kFDepth) * kFSlot + w * kS3Pitch;
        const float4 v = phase4(row, row - kS3Pitch, row + kS3Pitch, ld4s(Nb, lane), ld4s(Nt, lane), ld4s(F, lane), L,
                                x0, y, q, c2, lane);
        reinterpret_cast<float4*>(uout + ((int64_t)q * ny + y) * nx + xs)[lane] = v;
      }
    }
    if (!aborted) __syncthreads();  // the next task refills the slots
  }
  if (aborted && tid == 0) {
    atomicOr(err, 1u);  // the host reports FAS_ETIMEOUT
    for (int k = 0; k < kNBar3; ++k)
      if ((pend >> k) & 1u) mbar_wait_bounded(bar + k, (par >> k) & 1u, wait_ns);
  }
}

}  // namespace

bool sweep3d_supported(const LevelDesc<float>& L) {
  return L.nz > 1 && L.nx % kS3Cols == 0 && !L.varkappa && L.fax < 0 && L.per == 0 && L.ny >= 2 && L.nz >= 2;
}

cudaError_t sweep3d_prepare() {
  return cudaFuncSetAttribute(k_sweep3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kS3Smem);
}

cudaError_t launch_sweep3d(float* uout, const float* uin, const float* f, const LevelDesc<float>& L, int c1,
                           int sm_count, unsigned* err, unsigned long long wait_ns, int withhold, cudaStream_t stream) {
  // plane segments of 32..256 (four extra planes each) sized for about four tasks per block
  const int64_t cols = (int64_t)(L.nx / kS3Cols) * ((L.ny + kS3Rows - 1) / kS3Rows);
  const int64_t wave = (int64_t)sm_count * 2;
  const int64_t per = std::max<int64_t>(1, (wave * 4 + cols - 1) / cols);
  const int zseg = (int)std::min<int64_t>(256, std::max<int64_t>(32, (L.nz + per - 1) / per));
  const int64_t ntasks = cols * ((L.nz + zseg - 1) / zseg);
  const int blocks = (int)std::min<int64_t>(ntasks, wave);
  CUtensorMap tu, tf;
  cudaError_t e = tensor_map_3d(&tu, uin, sizeof(float), L.nx, L.ny, L.nz, kS3Pitch, kUTileRows, 1);
  if (e == cudaSuccess) e = tensor_map_3d(&tf, f, sizeof(float), L.nx, L.ny, L.nz, kS3Pitch, kFTileRows, 1);
  if (e != cudaSuccess) return e;
  k_sweep3d<<<blocks, kS3Threads, kS3Smem, stream>>>(uout, tu, tf, L, c1, zseg, err, wait_ns, withhold);
  return cudaGetLastError();
}

}  // namespace fasmg
