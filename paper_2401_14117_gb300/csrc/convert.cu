// convert.cu -- double <-> Posit(32,2) conversion and the element-wise
// Add/Sub/Mul/Div/Sqrt kernels (Sec. 4.2: r[i] = p[i] op q[i]).
//
// HBM-bound: 8+4 (from double), 4+8 (to double) or 4+4+4 bytes per element.
// Grid-stride loops over a grid of a few waves of the 152 SMs.
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
__global__ void elementwise_kernel(const uint32_t *__restrict__ p, const uint32_t *__restrict__ q,
                                   uint32_t *__restrict__ r, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    pz a = pz_decode(p[i]);
    pz out;
    if (OP == 4) {
      out = pz_sqrt(a);
    } else {
      pz b = pz_decode(q[i]);
      if (OP == 0) out = pz_add(a, b);
      else if (OP == 1) out = pz_sub(a, b);
      else if (OP == 2) out = pz_mul(a, b);
      else out = pz_div(a, b);
    }
    r[i] = pz_to_bits(out);
  }
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
  int g = grid_for(count);
  switch (op) {
    case 0: elementwise_kernel<0><<<g, kThreads, 0, stream>>>(p, q, r, count); break;
    case 1: elementwise_kernel<1><<<g, kThreads, 0, stream>>>(p, q, r, count); break;
    case 2: elementwise_kernel<2><<<g, kThreads, 0, stream>>>(p, q, r, count); break;
    case 3: elementwise_kernel<3><<<g, kThreads, 0, stream>>>(p, q, r, count); break;
    default: elementwise_kernel<4><<<g, kThreads, 0, stream>>>(p, p, r, count); break;
  }
  return launch_status();
}
