// convert.cu -- double <-> Posit(32,2) conversion and the element-wise
// Add/Sub/Mul/Div/Sqrt kernels (Sec. 4.2: r[i] = p[i] op q[i]).
//
// 8+4 (from double), 4+8 (to double) or 4+4+4 bytes per element; the
// element-wise operations cost 100 to 500 integer instructions per element,
// which makes them issue-bound rather than HBM-bound.  Grid-stride loops over
// a grid of a few waves of the 152 SMs.
#include "internal.cuh"

namespace posit {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t count) {
  int64_t blocks = ceil_div(count, kThreads);
  int64_t cap = 152 * 8;  // 8 resident blocks per SM at 256 threads
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

__global__ void from_double_kernel(const double *__restrict__ x, uint32_t *__restrict__ p,
                                   int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = pz_from_double(x[i]);
}

__global__ void to_double_kernel(const uint32_t *__restrict__ p, double *__restrict__ x,
                                 int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = pz_to_double(p[i]);
}

template <int OP>
__device__ __forceinline__ uint32_t elementwise_one(uint32_t x, uint32_t y) {
  pz a = pz_decode(x);
  pz out;
  if (OP == 4) {
    out = pz_sqrt(a);
  } else {
    pz b = pz_decode(y);
    if (OP == 0) out = pz_add(a, b);
    else if (OP == 1) out = pz_sub(a, b);
    else if (OP == 2) out = pz_mul(a, b);
    else out = pz_div(a, b);
  }
  return pz_to_bits(out);
}

// VEC: p, q and r are 16-byte aligned; four elements per thread and step
// with 128-bit loads and stores, then the count % 4 tail one by one.
template <int OP, bool VEC>
__global__ void elementwise_op_kernel(const uint32_t *__restrict__ p,
                                      const uint32_t *__restrict__ q, uint32_t *__restrict__ r,
                                      int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (VEC) {
    const int64_t n4 = count >> 2;
    const uint4 *p4 = reinterpret_cast<const uint4 *>(p);
    const uint4 *q4 = reinterpret_cast<const uint4 *>(q);
    uint4 *r4 = reinterpret_cast<uint4 *>(r);
    for (int64_t i = t0; i < n4; i += stride) {
      uint4 x = p4[i];
      uint4 y = OP == 4 ? x : q4[i];
      uint4 z;
      z.x = elementwise_one<OP>(x.x, y.x);
      z.y = elementwise_one<OP>(x.y, y.y);
      z.z = elementwise_one<OP>(x.z, y.z);
      z.w = elementwise_one<OP>(x.w, y.w);
      r4[i] = z;
    }
    done = n4 << 2;
  }
  for (int64_t i = done + t0; i < count; i += stride)
    r[i] = elementwise_one<OP>(p[i], OP == 4 ? 0u : q[i]);
}

template <int OP>
void launch_elementwise(const uint32_t *p, const uint32_t *q, uint32_t *r, int64_t count,
                        cudaStream_t stream) {
  const bool vec = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q) |
                     reinterpret_cast<uintptr_t>(r)) & 15u) == 0u;
  if (vec)
    elementwise_op_kernel<OP, true><<<grid_for(ceil_div(count, 4)), kThreads, 0, stream>>>(
        p, q, r, count);
  else
    elementwise_op_kernel<OP, false><<<grid_for(count), kThreads, 0, stream>>>(p, q, r, count);
}

}  // namespace
}  // namespace posit

using namespace posit;

extern "C" int posit_from_double(const double *x, posit32_t *p, int64_t count,
                                 cudaStream_t stream) {
  if (count < 0) return -3;
  if (count == 0) return POSIT_OK;
  if (!x) return -1;
  if (!p) return -2;
  from_double_kernel<<<grid_for(count), kThreads, 0, stream>>>(x, p, count);
  return launch_status();
}

extern "C" int posit_to_double(const posit32_t *p, double *x, int64_t count,
                               cudaStream_t stream) {
  if (count < 0) return -3;
  if (count == 0) return POSIT_OK;
  if (!p) return -1;
  if (!x) return -2;
  to_double_kernel<<<grid_for(count), kThreads, 0, stream>>>(p, x, count);
  return launch_status();
}

extern "C" int posit_elementwise(int op, const posit32_t *p, const posit32_t *q,
                                 posit32_t *r, int64_t count, cudaStream_t stream) {
  if (op < 0 || op > 4) return -1;
  if (count < 0) return -5;
  if (count == 0) return POSIT_OK;
  if (!p) return -2;
  if (op != 4 && !q) return -3;
  if (!r) return -4;
  switch (op) {
    case 0: launch_elementwise<0>(p, q, r, count, stream); break;
    case 1: launch_elementwise<1>(p, q, r, count, stream); break;
    case 2: launch_elementwise<2>(p, q, r, count, stream); break;
    case 3: launch_elementwise<3>(p, q, r, count, stream); break;
    default: launch_elementwise<4>(p, p, r, count, stream); break;
  }
  return launch_status();
}
