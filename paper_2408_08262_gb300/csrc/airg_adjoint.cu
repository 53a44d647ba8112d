// Adjoint form: the hierarchy of A^T (for the adjoint solve A^T lambda = g) and the sampled
// dense-dense product on A's pattern that gives dJ/dA = -lambda x^T.
#include "airg_common.cuh"

namespace airg {

// Deterministic CSR transpose: per-column counts, scan, scatter with atomic cursors, then each row
// of A^T sorted by column (the scatter order within a row is not deterministic, the sorted result
// is, because columns within a row are unique).
__global__ void k_tr_count(int n, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(cnt + ci[k], 1);
}
__global__ void k_tr_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                          const int* __restrict__ trp, int* __restrict__ cursor, int* __restrict__ tci,
                          double* __restrict__ tv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      const int p = trp[j] + atomicAdd(cursor + j, 1);
      tci[p] = (int)i;
      tv[p] = v[k];
    }
}
__global__ void k_sort_rows(int n, const int* __restrict__ rp, int* __restrict__ ci, double* __restrict__ v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = rp[i], e = rp[i + 1];
    for (int k = b + 1; k < e; ++k) {
      const int c = ci[k];
      const double x = v[k];
      int q = k - 1;
      while (q >= b && ci[q] > c) {
        ci[q + 1] = ci[q];
        v[q + 1] = v[q];
        --q;
      }
      ci[q + 1] = c;
      v[q + 1] = x;
    }
  }
}

int csr_transpose(const DCsr& A, DCsr& T, Arena& own, Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  AIRG_TRY(own.csr(T, A.ncols, A.nrows, A.nnz));
  int *cnt, *cursor;
  AIRG_TRY(tmp.alloc(&cnt, std::max(A.ncols, 1)));
  AIRG_TRY(tmp.alloc(&cursor, std::max(A.ncols, 1)));
  CU_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max(A.ncols, 1), s));
  CU_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * std::max(A.ncols, 1), s));
  if (n > 0) airg::note_launch(), k_tr_count<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, cnt);
  KERNEL_CHECK();
  AIRG_TRY(scan_i32(cnt, T.rp, A.ncols, tmp, s, nullptr));
  if (n > 0) airg::note_launch(), k_tr_fill<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, T.rp, cursor, T.ci, T.v);
  if (A.ncols > 0) airg::note_launch(), k_sort_rows<<<grid_for(A.ncols, 256), 256, 0, s>>>(A.ncols, T.rp, T.ci, T.v);
  KERNEL_CHECK();
  return AIRG_OK;
}

// out[k] = (scale * lam[i]) * x[col[k]] for every stored entry (i, col[k]) of the pattern.
__global__ void k_sddmm(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ lam,
                        const double* __restrict__ x, double scale, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double li = scale * lam[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) out[k] = li * x[ci[k]];
  }
}

}  // namespace airg

using namespace airg;

extern "C" int airg_transpose(const airg_csr* A, int32_t* rowptr_out, int32_t* col_out, double* val_out,
                              airg_stream_t stream) {
  if (!A || A->n < 0 || A->nnz < 0 || !rowptr_out || (A->nnz > 0 && (!col_out || !val_out))) return AIRG_ERR_ARG;
  if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))) return AIRG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp;
  tmp.s = s;
  DCsr D;
  D.nrows = D.ncols = A->n;
  D.nnz = A->nnz;
  D.rp = const_cast<int*>(A->rowptr);
  D.ci = const_cast<int*>(A->col);
  D.v = const_cast<double*>(A->val);
  int rc = validate_csr(D, tmp, s);
  if (rc == AIRG_OK) {
    Arena own;
    own.s = s;
    DCsr T;
    rc = csr_transpose(D, T, own, tmp, s);
    if (rc == AIRG_OK) rc = cuda_status(cudaMemcpyAsync(rowptr_out, T.rp, sizeof(int) * ((size_t)A->n + 1), cudaMemcpyDeviceToDevice, s));
    if (rc == AIRG_OK && A->nnz)
      rc = cuda_status(cudaMemcpyAsync(col_out, T.ci, sizeof(int) * (size_t)A->nnz, cudaMemcpyDeviceToDevice, s));
    if (rc == AIRG_OK && A->nnz)
      rc = cuda_status(cudaMemcpyAsync(val_out, T.v, sizeof(double) * (size_t)A->nnz, cudaMemcpyDeviceToDevice, s));
    own.release();
  }
  tmp.release();
  if (rc == AIRG_OK) rc = cuda_status(cudaStreamSynchronize(s));
  return rc;
}

extern "C" int airg_setup_transpose(const airg_csr* A, const airg_params* p, airg_stream_t stream,
                                    airg_hierarchy** out) {
  if (!out || !A || !p || A->n <= 0 || A->nnz < 0) return AIRG_ERR_ARG;
  *out = nullptr;
  if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return AIRG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp, own;
  tmp.s = own.s = s;
  DCsr D;
  D.nrows = D.ncols = A->n;
  D.nnz = A->nnz;
  D.rp = const_cast<int*>(A->rowptr);
  D.ci = const_cast<int*>(A->col);
  D.v = const_cast<double*>(A->val);
  int rc = validate_csr(D, tmp, s);
  DCsr T;
  if (rc == AIRG_OK) rc = csr_transpose(D, T, own, tmp, s);
  if (rc == AIRG_OK) {
    airg_csr At{T.nrows, T.nnz, T.rp, T.ci, T.v};
    rc = airg_setup(&At, p, stream, out);  // copies the matrix; synchronises the stream
  }
  cudaStreamSynchronize(s);
  own.release();
  tmp.release();
  return rc;
}

extern "C" int airg_sddmm(const airg_csr* pattern, const double* lam, const double* x, double scale, double* out_val,
                          airg_stream_t stream) {
  if (!pattern || pattern->n < 0 || pattern->nnz < 0 || !lam || !x || (pattern->nnz > 0 && !out_val)) return AIRG_ERR_ARG;
  if (pattern->n > 0 && (!pattern->rowptr || (pattern->nnz > 0 && !pattern->col))) return AIRG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (pattern->n > 0)
    airg::note_launch(), k_sddmm<<<grid_for(pattern->n, 256), 256, 0, s>>>(pattern->n, pattern->rowptr, pattern->col, lam,
                                                                          x, scale, out_val);
  return cuda_status(cudaGetLastError());
}
