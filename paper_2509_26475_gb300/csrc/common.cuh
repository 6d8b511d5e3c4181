// Device helpers shared by the phicomb kernels: bounded grid barrier, cross-block max slots,
// scaled sums of squares and vector loads for the row-major block tiles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "phicomb.h"

namespace phic {

constexpr int kBlock = 256;  // threads per block of every persistent kernel

// Control block at the head of each persistent kernel's workspace region; zeroed before launch.
struct __align__(256) Ctl {
  unsigned long long bar;  // team-barrier arrivals since launch (monotone: epoch e completes at e * team size)
  int status;              // first phic_status != OK seen by any block
  int fault;               // unused padding kept for layout stability
  unsigned long long slot[4][4];  // max-reduction slots (bit patterns of non-negative values), by phase % 4
  int dia_keys[16];        // set of the operator's diagonal offsets (offset + n; 0 = empty), hashed
  int dia_ovf;             // more than 16 distinct offsets
  int pad[9];
};
static_assert(sizeof(Ctl) == 256, "Ctl is one 256-byte line");

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_status(Ctl* c, int st) { atomicCAS(&c->status, 0, st); }

__device__ __forceinline__ int read_status(const Ctl* c) { return *(volatile const int*)&c->status; }

__device__ __forceinline__ void bar_arrive(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long bar_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The CTAs that work on one problem instance together: the whole grid of a single-instance launch, or
// a subset of a batched launch.  `rank` and `size` replace blockIdx.x and gridDim.x inside the method's
// kernels; `ctl` is the instance's control block (zeroed before the launch); thread 0 of each member keeps
// `epoch`, the number of team barriers it has passed in this launch.
struct Team {
  Ctl* ctl;
  int rank, size;
  unsigned long long spin_ns;
  unsigned long long epoch;
};

__device__ __forceinline__ Team grid_team(Ctl* c, unsigned long long spin_ns) {
  return Team{c, (int)blockIdx.x, (int)gridDim.x, spin_ns, 0ull};
}

// Team barrier with leader work on both sides.  Every thread of every member calls it.  Thread 0 runs
// pre() after its block's threads have arrived (their writes are visible to it) and before it signals
// arrival with a release reduction on the monotone counter; it then polls the counter with acquire loads
// until every member has arrived (epoch * size arrivals), runs post() (reads the team's results, decides,
// writes shared memory) and releases the block.  The release/acquire pair orders every write made
// before the barrier by any thread of the team before every read after it.  A wait longer than spin_ns
// sets PHIC_TIMEOUT and returns false in every thread of the block that gave up; the caller then leaves
// the instance, so no block ever waits without bound.
template <typename Pre, typename Post>
__device__ __forceinline__ bool team_sync_lead(Team& tm, Pre&& pre, Post&& post) {
  __shared__ int s_ok2;
  __syncthreads();
  if (threadIdx.x == 0) {
    pre();
    int ok = 1;
    tm.epoch += 1;
    if (tm.size > 1) {
      const unsigned long long target = tm.epoch * (unsigned long long)tm.size;
      bar_arrive(&tm.ctl->bar);
      if (bar_load(&tm.ctl->bar) < target) {
        const unsigned long long t0 = global_ns();
        unsigned spins = 0;
        while (bar_load(&tm.ctl->bar) < target) {
          if ((++spins & 31u) == 0 && global_ns() - t0 > tm.spin_ns) {
            ok = 0;
            set_status(tm.ctl, PHIC_TIMEOUT);
            break;
          }
        }
      }
    } else {
      __threadfence();
    }
    if (ok) post();
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

// As team_sync_lead, but post() runs in every lane of warp 0 (lane 0 still signals the arrival and waits).
// On GB300 an FP64 instruction occupies the FP64 pipe for a whole warp however few of its lanes are
// active, so scalar FP64 work for several combinations is spread over the lanes, one combination each,
// and costs what one combination costs.  The lanes see the other members' writes after lane 0's acquire
// through the warp barrier, as the block's threads do after the block barrier.
// prep() runs first, in every lane of warp 0: loads issued there (say, of the next term's constants) travel
// while lane 0 waits, and post() finds them in registers.
template <typename Prep, typename Pre, typename Post>
__device__ __forceinline__ bool team_sync_lead_w(Team& tm, Prep&& prep, Pre&& pre, Post&& post) {
  __shared__ int s_ok3;
  __syncthreads();
  if (threadIdx.x < 32) {
    int ok = 1;
    prep();
    if (threadIdx.x == 0) {
      pre();
      tm.epoch += 1;
      if (tm.size > 1) {
        const unsigned long long target = tm.epoch * (unsigned long long)tm.size;
        bar_arrive(&tm.ctl->bar);
        if (bar_load(&tm.ctl->bar) < target) {
          const unsigned long long t0 = global_ns();
          unsigned spins = 0;
          while (bar_load(&tm.ctl->bar) < target) {
            if ((++spins & 31u) == 0 && global_ns() - t0 > tm.spin_ns) {
              ok = 0;
              set_status(tm.ctl, PHIC_TIMEOUT);
              break;
            }
          }
        }
      } else {
        __threadfence();
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) post();
    __syncwarp();
    if (threadIdx.x == 0) s_ok3 = ok;
  }
  __syncthreads();
  return s_ok3 != 0;
}

__device__ __forceinline__ bool team_sync(Team& tm) {
  return team_sync_lead(tm, [] {}, [] {});
}

// ---- max over the grid of non-negative doubles, carried as their bit patterns --------------------
// Non-negative doubles order like their unsigned bit patterns; NaN and Inf patterns sort above every
// finite value, so a non-finite norm anywhere surfaces in the slot.
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long u) { return __longlong_as_double((long long)u); }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Block-wide max of per-thread values; the result is valid in thread 0.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v) {
  __shared__ unsigned long long s_w[kBlock / 32];
  v = warp_max_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < kBlock / 32 ? s_w[lane] : 0ull;
    v = warp_max_u64(v);
  }
  return v;
}

// Slots of phase p + 2 are cleared by the team's rank 0 during phase p (every member has read them in
// phase p - 2 before arriving at barrier p - 1, and writes them only after barrier p + 1).
__device__ __forceinline__ void slot_reset(const Team& tm, int phase) {
  if (tm.rank == 0 && threadIdx.x < 4) tm.ctl->slot[(phase + 2) & 3][threadIdx.x] = 0ull;
}
__device__ __forceinline__ void slot_max(Ctl* c, int phase, int idx, unsigned long long v) {
  atomicMax(&c->slot[phase & 3][idx], v);
}
__device__ __forceinline__ double slot_get(const Ctl* c, int phase, int idx) {
  return bitsd(*(volatile const unsigned long long*)&c->slot[phase & 3][idx]);
}

// ---- scaled sum of squares: value = ssq * 2^(2e) ------------------------------------------------
// The power-of-two scalings move the exponent field with integer operations (exact; on GB300 FP64
// instructions are scarce), so adding an element costs one FP64 fused multiply-add.
struct Ssq {
  int e;
  double ssq;
};
constexpr int kSsqEmpty = -4000;
constexpr int kSsqNonfinite = 5000;

__device__ __forceinline__ Ssq ssq_empty() { return Ssq{kSsqEmpty, 0.0}; }

// x 2^-d for a finite normal x whose scaled exponent stays at most 1023; results under 2^-998 flush
// to 0 (they lie at least 2^-998 below the running scale, so their squares cannot change the sum).
__device__ __forceinline__ double pow2_down(double x, int d) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex - d <= 25) return 0.0;
  return __longlong_as_double(b - (long long)d * 4503599627370496LL);  // d * 2^52
}

__device__ __forceinline__ void ssq_add(Ssq& a, double x) {
  const long long b = __double_as_longlong(x);
  const int bex = (int)((b >> 52) & 0x7ff);
  if (bex == 0) return;  // zero or subnormal: below 2^-1022, negligible against any normal element
  if (bex == 0x7ff) {    // Inf or NaN: keep it visible
    a.e = kSsqNonfinite;
    a.ssq = (double)NAN;
    return;
  }
  if (a.e >= kSsqNonfinite) return;
  const int ex = bex - 1023;
  if (ex > a.e) {
    a.ssq = (a.e == kSsqEmpty) ? 0.0 : pow2_down(a.ssq, 2 * (ex - a.e));
    a.e = ex;
  }
  const double y = pow2_down(x, a.e);  // x 2^-e, exponent at most 0
  a.ssq = fma(y, y, a.ssq);
}

__device__ __forceinline__ Ssq ssq_combine(Ssq a, Ssq b) {
  if (a.e == kSsqEmpty) return b;
  if (b.e == kSsqEmpty) return a;
  if (a.e >= kSsqNonfinite || b.e >= kSsqNonfinite) return Ssq{kSsqNonfinite, (double)NAN};
  const int e = a.e > b.e ? a.e : b.e;
  return Ssq{e, pow2_down(a.ssq, 2 * (e - a.e)) + pow2_down(b.ssq, 2 * (e - b.e))};
}

// log of the 2-norm; -inf for a zero vector, NaN when a non-finite value was seen.
__device__ __forceinline__ double ssq_log_norm(Ssq a) {
  if (a.e == kSsqEmpty || a.ssq == 0.0) return -INFINITY;
  if (a.e >= kSsqNonfinite) return (double)NAN;
  return (double)a.e * 0.69314718055994530942 + 0.5 * log(a.ssq);
}

__device__ __forceinline__ Ssq warp_ssq(Ssq a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Ssq b;
    b.e = __shfl_xor_sync(0xffffffffu, a.e, o);
    b.ssq = __shfl_xor_sync(0xffffffffu, a.ssq, o);
    a = ssq_combine(a, b);
  }
  return a;
}

// Block-wide combine; the result is valid in thread 0.
__device__ __forceinline__ Ssq block_ssq(Ssq a) {
  __shared__ int s_e[kBlock / 32];
  __shared__ double s_s[kBlock / 32];
  a = warp_ssq(a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    s_e[wid] = a.e;
    s_s[wid] = a.ssq;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < kBlock / 32 ? Ssq{s_e[lane], s_s[lane]} : ssq_empty();
    a = warp_ssq(a);
  }
  return a;
}

// ---- vector loads/stores of CW consecutive elements (the tiles keep them aligned) ----------------
template <typename T, int CW>
struct VecIO;

template <>
struct VecIO<double, 1> {
  static __device__ __forceinline__ void ld(const double* p, double (&x)[1]) { x[0] = *p; }
  static __device__ __forceinline__ void st(double* p, const double (&x)[1]) { *p = x[0]; }
};
template <>
struct VecIO<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&x)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  }
};
template <>
struct VecIO<double, 4> {
  static __device__ __forceinline__ void ld(const double* p, double (&x)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&x)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  }
};
// Three and five values a lane (series tiles whose width is a multiple of 3 or 5, so that a row needs no
// idle lanes): such chunks are aligned to one element only, so they move one element at a time.
template <typename T, int CW>
struct VecIOScalar {
  static __device__ __forceinline__ void ld(const T* p, T (&x)[CW]) {
#pragma unroll
    for (int j = 0; j < CW; ++j) x[j] = p[j];
  }
  static __device__ __forceinline__ void st(T* p, const T (&x)[CW]) {
#pragma unroll
    for (int j = 0; j < CW; ++j) p[j] = x[j];
  }
};
template <>
struct VecIO<double, 3> : VecIOScalar<double, 3> {};
template <>
struct VecIO<double, 5> : VecIOScalar<double, 5> {};
template <>
struct VecIO<float, 3> : VecIOScalar<float, 3> {};
template <>
struct VecIO<float, 5> : VecIOScalar<float, 5> {};
template <>
struct VecIO<float, 1> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[1]) { x[0] = *p; }
  static __device__ __forceinline__ void st(float* p, const float (&x)[1]) { *p = x[0]; }
};
template <>
struct VecIO<float, 2> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[2]) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void st(float* p, const float (&x)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
  }
};
template <>
struct VecIO<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
};

template <>
struct VecIO<float, 8> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&x)[8]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
  }
};

// Loads and stores of the workspace tiles, which are always in global memory.  An FP32 lane's 32-byte
// chunk (8 floats) moves as one 256-bit access (sm_100 and later) instead of two 128-bit ones: the
// 1024^2 FP32 recovery, latency-bound on L2, went 86.1 -> 74.3 ms for 2882 terms on GB300.  The same for
// 4-double chunks measured 1.3 % slower on the FP64 recovery (bound by the FP64 pipe), so FP64 keeps
// VecIO.  The chunks are 32-byte aligned: tiles start on 256-byte boundaries and their row strides and
// chunk offsets are multiples of the chunk.  Plain (coherent) accesses: the tiles are rewritten between
// the terms of one launch.  Volatile, so that no load is merged with or moved across another access of
// the same kind; E, which may live in shared memory, keeps VecIO.
template <typename T, int CW>
struct VecIOG : VecIO<T, CW> {};
template <>
struct VecIOG<float, 8> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[8]) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p));
  }
  static __device__ __forceinline__ void st(float* p, const float (&x)[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "f"(x[0]), "f"(x[1]), "f"(x[2]), "f"(x[3]), "f"(x[4]), "f"(x[5]), "f"(x[6]), "f"(x[7])
                 : "memory");
  }
};

// Sum over the lanes of one row group (Lp2 consecutive lanes, a power of two <= 32, aligned).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int Lp2) {
  for (int o = 1; o < Lp2; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace phic
