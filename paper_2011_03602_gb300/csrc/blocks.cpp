// Code-pattern table for function-block offload (Sec. 3.2.2, Sec. 4.2.1).
//
// The paper matches the names of library calls found in the source against
// a code-pattern database and swaps matching calls for GPU implementations
// (a matrix product, a Fourier transform).  Here the database is a small
// static table of common CPU entry points per source language; a match
// yields the block id of the GPU replacement behind this library's ABI.
#include <cstring>

#include "oo_internal.h"

namespace oo {

namespace {
struct Entry {
    int lang;
    const char *name;
    int block;
};

const Entry kTable[] = {
    // C / C++ (BLAS, FFTW, GSL)
    {OO_LANG_C, "cblas_dgemm", OO_BLOCK_GEMM},
    {OO_LANG_C, "dgemm_", OO_BLOCK_GEMM},
    {OO_LANG_C, "dgemm", OO_BLOCK_GEMM},
    {OO_LANG_C, "gsl_blas_dgemm", OO_BLOCK_GEMM},
    {OO_LANG_C, "fftw_plan_dft_1d", OO_BLOCK_FFT},
    {OO_LANG_C, "fftw_execute", OO_BLOCK_FFT},
    {OO_LANG_C, "gsl_fft_complex_forward", OO_BLOCK_FFT},
    {OO_LANG_C, "gsl_fft_complex_radix2_forward", OO_BLOCK_FFT},
    // Python (NumPy, SciPy)
    {OO_LANG_PYTHON, "numpy.dot", OO_BLOCK_GEMM},
    {OO_LANG_PYTHON, "numpy.matmul", OO_BLOCK_GEMM},
    {OO_LANG_PYTHON, "numpy.ndarray.dot", OO_BLOCK_GEMM},
    {OO_LANG_PYTHON, "scipy.linalg.blas.dgemm", OO_BLOCK_GEMM},
    {OO_LANG_PYTHON, "numpy.fft.fft", OO_BLOCK_FFT},
    {OO_LANG_PYTHON, "numpy.fft.ifft", OO_BLOCK_FFT},
    {OO_LANG_PYTHON, "scipy.fft.fft", OO_BLOCK_FFT},
    {OO_LANG_PYTHON, "scipy.fftpack.fft", OO_BLOCK_FFT},
    // Java (Apache Commons Math, JTransforms, EJML)
    {OO_LANG_JAVA, "org.apache.commons.math3.linear.RealMatrix.multiply", OO_BLOCK_GEMM},
    {OO_LANG_JAVA, "org.apache.commons.math3.linear.Array2DRowRealMatrix.multiply", OO_BLOCK_GEMM},
    {OO_LANG_JAVA, "org.ejml.dense.row.CommonOps_DDRM.mult", OO_BLOCK_GEMM},
    {OO_LANG_JAVA, "org.jtransforms.fft.DoubleFFT_1D.complexForward", OO_BLOCK_FFT},
    {OO_LANG_JAVA, "org.jtransforms.fft.DoubleFFT_1D.complexInverse", OO_BLOCK_FFT},
    {OO_LANG_JAVA, "org.apache.commons.math3.transform.FastFourierTransformer.transform",
     OO_BLOCK_FFT},
};
}  // namespace

int lookup_block(const char *callee, int lang) {
    for (const auto &e : kTable)
        if (e.lang == lang && std::strcmp(e.name, callee) == 0) return e.block;
    return 0;
}

}  // namespace oo
