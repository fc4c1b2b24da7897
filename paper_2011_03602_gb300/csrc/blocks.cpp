// Code-pattern table for function-block offload (Sec. 3.2.2, Sec. 4.2.1).
//
// The paper matches the names of library calls found in the source against
// a code-pattern database and swaps matching calls for GPU implementations
// (a matrix product, a Fourier transform).  Here the database is a small
// static table of common CPU entry points per source language; a match
// yields the block id of the GPU replacement behind this library's ABI.
#include <cstring>
#include <string>

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

namespace {
int exact(const std::string &name, int lang) {
    for (const auto &e : kTable)
        if (e.lang == lang && name == e.name) return e.block;
    return 0;
}

// Spelling variants of one call the code analysis may report: import
// aliases (np, sp, la), module re-exports, a Java class used without its
// package, case of Fortran-style BLAS names.  Each maps to the spelling in
// the table; nothing here guesses at code it has not seen (similarity
// detection of hand-written blocks is a separate tool).
std::string canonical(std::string name, int lang) {
    auto replace_prefix = [&](const char *from, const char *to) {
        const size_t n = std::strlen(from);
        if (name.compare(0, n, from) == 0) name = std::string(to) + name.substr(n);
    };
    if (lang == OO_LANG_PYTHON) {
        replace_prefix("np.", "numpy.");
        replace_prefix("sp.", "scipy.");
        replace_prefix("la.", "scipy.linalg.");
        replace_prefix("scipy.fft._basic.", "scipy.fft.");
        replace_prefix("numpy.core.multiarray.", "numpy.");
        replace_prefix("numpy.core.numeric.", "numpy.");
    } else if (lang == OO_LANG_C) {
        std::string low;
        for (char ch : name) low += (char)((ch >= 'A' && ch <= 'Z') ? ch - 'A' + 'a' : ch);
        if (low == "dgemm" || low == "dgemm_") name = low;
    }
    return name;
}
}  // namespace

int lookup_block(const char *callee, int lang) {
    const std::string name(callee);
    if (int b = exact(name, lang)) return b;
    if (int b = exact(canonical(name, lang), lang)) return b;
    if (lang == OO_LANG_JAVA && name.find('.') != std::string::npos) {
        // Class.method without its package: unique suffix match in the table
        int found = 0, count = 0;
        for (const auto &e : kTable) {
            if (e.lang != OO_LANG_JAVA) continue;
            const std::string full(e.name);
            if (full.size() > name.size() && full.compare(full.size() - name.size(), name.size(), name) == 0 &&
                full[full.size() - name.size() - 1] == '.') {
                found = e.block;
                ++count;
            }
        }
        if (count >= 1) {
            // several matches are fine only if they agree on the block
            for (const auto &e : kTable) {
                if (e.lang != OO_LANG_JAVA) continue;
                const std::string full(e.name);
                if (full.size() > name.size() && full.compare(full.size() - name.size(), name.size(), name) == 0 &&
                    full[full.size() - name.size() - 1] == '.' && e.block != found)
                    return 0;
            }
            return found;
        }
    }
    return 0;
}

}  // namespace oo
