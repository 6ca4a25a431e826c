// Device helpers of the batched step: small vector algebra, shared-memory
// layout of a group of 32 environments, and the launch table.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "brax_params.h"

namespace brax {

#define BRAX_MAX_SEGS 8

// Constant-memory pool holding the parameter blobs of all live systems.  A
// warp reads its body's parameters with a warp-uniform index, so the loads go
// through the constant cache and the uniform datapath, not the LSU.
constexpr int kPoolBytes = 61440;

// One system's share of a launch.  A thread block runs G groups of 32
// environments of one system; group g's warps are bodies 0..B-1 (warp =
// body, lane = environment).
struct Seg {
  const unsigned char* blob;  // device copy of the parameter blob (default_qp)
  int32_t pool_off;           // offset of the blob in the constant parameter pool
  int32_t blob_bytes;
  int32_t B, P, A;
  int32_t groups;  // groups of 32 environments per thread block
  int32_t cta_begin, cta_end;
  int64_t n_envs;
  const float* state0;
  const float* actions;
  float* state_T;
  float* ckpt;
  float* torso;
  int32_t* ccount;
  int32_t* status;
  // gym-like environment layer (brax_env_rollout; obs == nullptr: off)
  float* obs;                 // [T, N, obs_dim] after every step, before any reset
  float* reward;              // [T, N]
  uint8_t* done;              // [T, N]
  const float* reset_state;   // [N, B, 13]: a done environment continues from here
  int32_t obs_dim, auto_reset;
  float fwd_w_dt;             // forward_weight / dt
  float healthy, ctrl_cost, min_z, max_z;
  int32_t ck_stage;  // 1: the paired kernel stages checkpoints in shared memory (after its groups)
  // backward
  const float* g_state_T;
  const float* g_torso;
  float* g_actions;
  float* g_state0;
  float* ws;  // per-segment workspace
};

// Chunked schedule of a persistent rollout.  A block keeps its environments
// on chip for the whole rollout, so when the blocks of a launch are not a
// whole number of resident waves the last wave runs part-empty from the first
// step to the last.  Instead the rollout of each block-sized unit of
// environments is cut into n_chunks chunks of chunk_steps steps: the launch
// has one block per (chunk, unit) item, and a block takes its item from a
// counter when it starts, so items run in the order blocks start, chunk-major;
// chunk c of a unit continues from the state that chunk c-1 left in state_T,
// once the unit's flag says chunk c-1 is done.  A block that holds item i
// started after the blocks holding items < i, so every wait ends.
// sched[0] is the counter, sched[1] an abort flag (set by a block whose wait
// gave up, so that later blocks stop at once), sched[32 + u] the flag of unit
// u (chunks done); all start at zero.  n_chunks = 0: block i runs unit i for
// the whole rollout.
struct Sched {
  int32_t n_chunks = 0;
  int32_t chunk_steps = 0;
  int32_t n_units = 0;
  int32_t first_item = 0;     // first item the counter hands out (0 except in the wait test)
  int32_t* sched = nullptr;
  int64_t wait_ns = 0;        // a wait for a flag gives up after this long (BRAX_ERR_TIMEOUT)
};

struct Launch {
  int32_t n_segs;
  int32_t T, K;
  int32_t pad;
  Seg seg[BRAX_MAX_SEGS];
  Sched sc;
};

// Status bits a kernel ORs into Seg::status (brax_sync_status reports them).
constexpr int32_t kStatusNonfinite = 1, kStatusTimeout = 2;

__device__ __forceinline__ int32_t load_acquire(const int32_t* p) {
  int32_t x;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
  return x;
}
__device__ __forceinline__ void store_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0's part of starting a block under a chunked schedule: take the
// block's item (the next ticket of the counter) and wait until the unit's
// previous chunk is done.  Returns the item; n_items when there is none for
// this block; -1 when the schedule was aborted; -2 when this wait gave up
// after wait_ns nanoseconds of the global timer (it then sets the abort flag;
// the caller reports kStatusTimeout).  *ticket is the ticket taken.
__device__ __forceinline__ int take_item(const Sched& sc, int n_items, int* ticket) {
  const int it = sc.first_item + atomicAdd(sc.sched, 1);
  *ticket = it;
  if (it >= n_items) return n_items;
  if (it < sc.n_units) return it;  // chunk 0 waits for nothing
  const int32_t* flag = sc.sched + 32 + it % sc.n_units;
  const int32_t need = it / sc.n_units;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (load_acquire(flag) >= need) return it;
    if (load_acquire(sc.sched + 1) != 0) return -1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if ((int64_t)(t - t0) > sc.wait_ns) {
      atomicExch(sc.sched + 1, 1);
      return -2;
    }
    __nanosleep(200);
  }
}

// ------------------------------------------------------------------ algebra
struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 mk3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return V3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// c + a x b with each component one multiply and two fused multiply-adds
__device__ __forceinline__ V3 cross_add(V3 a, V3 b, V3 c) {
  return V3{fmaf(a.y, b.z, fmaf(-a.z, b.y, c.x)), fmaf(a.z, b.x, fmaf(-a.x, b.z, c.y)),
            fmaf(a.x, b.y, fmaf(-a.y, b.x, c.z))};
}
__device__ __forceinline__ V3 fma3(float s, V3 a, V3 b) {  // s*a + b
  return V3{fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)};
}
__device__ __forceinline__ V3 ld3(const float* p) { return V3{p[0], p[1], p[2]}; }

// Row-major 3x3.
struct M3 {
  float m[9];
};
__device__ __forceinline__ V3 mul(const M3& R, V3 o) {
  return V3{fmaf(R.m[0], o.x, fmaf(R.m[1], o.y, R.m[2] * o.z)), fmaf(R.m[3], o.x, fmaf(R.m[4], o.y, R.m[5] * o.z)),
            fmaf(R.m[6], o.x, fmaf(R.m[7], o.y, R.m[8] * o.z))};
}
__device__ __forceinline__ V3 mulT(const M3& R, V3 o) {
  return V3{fmaf(R.m[0], o.x, fmaf(R.m[3], o.y, R.m[6] * o.z)), fmaf(R.m[1], o.x, fmaf(R.m[4], o.y, R.m[7] * o.z)),
            fmaf(R.m[2], o.x, fmaf(R.m[5], o.y, R.m[8] * o.z))};
}
__device__ __forceinline__ V3 mulc(const M3& R, const float* o) { return mul(R, ld3(o)); }

// Rotation matrix of a unit quaternion (w, x, y, z), body to world.
__device__ __forceinline__ M3 qmat(float qw, float qx, float qy, float qz) {
  const float x2 = qx + qx, y2 = qy + qy, z2 = qz + qz;
  M3 R;
  R.m[0] = fmaf(-qy, y2, fmaf(-qz, z2, 1.f));
  R.m[1] = fmaf(qx, y2, -qw * z2);
  R.m[2] = fmaf(qx, z2, qw * y2);
  R.m[3] = fmaf(qx, y2, qw * z2);
  R.m[4] = fmaf(-qx, x2, fmaf(-qz, z2, 1.f));
  R.m[5] = fmaf(qy, z2, -qw * x2);
  R.m[6] = fmaf(qx, z2, -qw * y2);
  R.m[7] = fmaf(qy, z2, qw * x2);
  R.m[8] = fmaf(-qx, x2, fmaf(-qy, y2, 1.f));
  return R;
}

// Symmetric 3x3 (xx, xy, xz, yy, yz, zz): world inverse inertia R diag(d) R^T.
struct S6 {
  float a[6];
};
__device__ __forceinline__ S6 inv_inertia_world(const M3& R, const float* d) {
  S6 s;
  const float r00 = R.m[0] * d[0], r01 = R.m[1] * d[1], r02 = R.m[2] * d[2];
  const float r10 = R.m[3] * d[0], r11 = R.m[4] * d[1], r12 = R.m[5] * d[2];
  s.a[0] = fmaf(r00, R.m[0], fmaf(r01, R.m[1], r02 * R.m[2]));
  s.a[1] = fmaf(r00, R.m[3], fmaf(r01, R.m[4], r02 * R.m[5]));
  s.a[2] = fmaf(r00, R.m[6], fmaf(r01, R.m[7], r02 * R.m[8]));
  s.a[3] = fmaf(r10, R.m[3], fmaf(r11, R.m[4], r12 * R.m[5]));
  s.a[4] = fmaf(r10, R.m[6], fmaf(r11, R.m[7], r12 * R.m[8]));
  const float r20 = R.m[6] * d[0], r21 = R.m[7] * d[1], r22 = R.m[8] * d[2];
  s.a[5] = fmaf(r20, R.m[6], fmaf(r21, R.m[7], r22 * R.m[8]));
  return s;
}
__device__ __forceinline__ V3 mul(const S6& s, V3 v) {
  return V3{fmaf(s.a[0], v.x, fmaf(s.a[1], v.y, s.a[2] * v.z)), fmaf(s.a[1], v.x, fmaf(s.a[3], v.y, s.a[4] * v.z)),
            fmaf(s.a[2], v.x, fmaf(s.a[4], v.y, s.a[5] * v.z))};
}

// Frozen-axis masks: bit i of `bits` freezes axis i.
__device__ __forceinline__ V3 mask3(uint32_t bits, V3 a) {
  return V3{(bits & 1u) ? 0.f : a.x, (bits & 2u) ? 0.f : a.y, (bits & 4u) ? 0.f : a.z};
}

__device__ __forceinline__ float clamp1(float a) { return fminf(fmaxf(a, -1.f), 1.f); }

// Four-quadrant arctangent in (-pi, pi]: octant reduction to a = min/max in
// [0, 1], atan(a) ~ a P(a^2) with P of degree 7, then the octant undone.
// atan2(0, 0) = 0.  P was fitted for this library in FP64 by iteratively
// reweighted least squares on the relative error over 20,001 Chebyshev nodes
// of [0, 1] (a Lawson-style minimax fit); evaluated in FP32 Horner form its
// error is at most 1.3e-7 rad on [0, 1].
__device__ __forceinline__ float fast_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  const float s = a * a;
  float p = -0.004037295f;
  p = fmaf(p, s, 0.021790044f);
  p = fmaf(p, s, -0.055787466f);
  p = fmaf(p, s, 0.096311055f);
  p = fmaf(p, s, -0.13903217f);
  p = fmaf(p, s, 0.19945158f);
  p = fmaf(p, s, -0.3332969f);
  p = fmaf(p, s, 0.9999993f);
  float r = a * p;
  if (ay > ax) r = 1.5707963267948966f - r;
  if (x < 0.f) r = 3.141592653589793f - r;
  return copysignf(r, y);
}

// Named barrier for one group of warps (id 1..15; id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Producer side of a named barrier: mark arrival without waiting.
__device__ __forceinline__ void bar_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------------ group shared memory
// Four consecutive fields of one lane form one float4, so a warp moves a
// chunk with one 16-byte access per lane (512 contiguous bytes, no bank
// conflict) instead of four scalar accesses.
// pub  [B][6][32] float4: a publishing body's post-kinematic
//                         (x, R0) (R1..R4) (R5..R8) (v, w.x) (w.y, w.z, Ii0, Ii1) (Ii2..Ii5)
// react[B][2][32] float4: a child's joint reaction on its parent (F, tau.x) (tau.y, tau.z, -, -)
// slot [P][2][32] float4: a body-body pair's (J, p.x) (p.y, p.z, active flag, -)
struct GroupMem {
  float4* pub;
  float4* react;
  float4* slot;
  int* cnt;
  __device__ __forceinline__ float4* pub4(int b, int c) { return pub + (b * (kPubFields / 4) + c) * 32; }
  __device__ __forceinline__ float4* react4(int b, int c) { return react + (b * (kReactFields / 4) + c) * 32; }
  __device__ __forceinline__ float4* slot4(int k, int c) { return slot + (k * (kSlotFields / 4) + c) * 32; }
};
// base must be 16-byte aligned.
__device__ __forceinline__ GroupMem group_mem(float* base, int B, int P) {
  GroupMem m;
  m.pub = reinterpret_cast<float4*>(base);
  m.react = m.pub + B * (kPubFields / 4) * 32;
  m.slot = m.react + B * (kReactFields / 4) * 32;
  m.cnt = reinterpret_cast<int*>(m.slot + P * (kSlotFields / 4) * 32);
  return m;
}
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ void st2(float4* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ float2 ld2(const float4* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 ld2hi(const float4* p) { return *(reinterpret_cast<const float2*>(p) + 1); }

}  // namespace brax
