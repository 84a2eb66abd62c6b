// Batched dense kernels for the BDDC set-up: variable-size batched GEMM and
// in-place blocked Gauss-Jordan inversion of SPD matrices (no pivoting; SPD
// matrices are Jacobi-scaled before inversion).  Row-major storage, leading
// dimensions padded to multiples of 4 elements.
#pragma once

#include "ufe_internal.cuh"

namespace ufe {

struct GemmDesc {
  int m, n, k;
  int lda, ldb, ldc;
  int64_t a, b, c;   // element offsets into the A, B, C base pointers
};

struct InvDesc {
  int n, ld;
  int64_t off;
};

// C = alpha * op(A) op(B) + beta * C for every descriptor; trans flags select op.
template <typename T>
void batched_gemm(bool transA, bool transB, const std::vector<GemmDesc>& descs, const T* A, const T* B, T* C,
                  T alpha, T beta, cudaStream_t s);

// in-place inverse of each SPD matrix; status[b] |= DEV_SINGULAR on a non-positive
// pivot, |= DEV_ILLCOND on a pivot below pivot_floor (0: no test)
template <typename T>
void batched_inverse(const std::vector<InvDesc>& descs, T* base, int* status, cudaStream_t s, T pivot_floor = T(0));

// FP32 inversions use the tensor-core (3xTF32) update unless the environment variable
// UFE_FP32_GJ is "simt" (the SIMT update, kept for comparison)
bool fp32_tensor_cores();

// in-place inverse of one large SPD matrix using the whole GPU; first_col (optional,
// host) holds for every row the first column with a nonzero, and the steps then skip
// the blocks outside the matrix's envelope
template <typename T>
void large_inverse(T* A, int n, int ld, int* status, cudaStream_t s, const std::vector<int32_t>* first_col = nullptr);

}  // namespace ufe
