// The Java front-end of the offload library (Sec. 3.3.3, Sec. 4.3.3): a
// Java program's function blocks and loop patterns reach the same C ABI as
// the C and Python front-ends, through the JNI shim in oo_jni.c.
//
// Build (needs a JDK; none is installed on the build or GPU machines here):
//   javac -h . OoNative.java
//   gcc -shared -fPIC -I$JAVA_HOME/include -I$JAVA_HOME/include/linux \
//       -I../../../include oo_jni.c -L.. -loo -o liboo_jni.so
package oo;

public final class OoNative {
    static { System.loadLibrary("oo_jni"); }

    public static final int BLOCK_GEMM = 1, BLOCK_FFT = 2, BLOCK_JACOBI = 3;
    public static final int LANG_JAVA = 2;

    /** Returns a context handle; throws on failure. */
    public static native long create(int device);
    public static native void destroy(long ctx);
    /** Code-pattern lookup of a callee name for Java sources; 0 when absent. */
    public static native int lookupBlock(String callee);
    /** C = A B (row-major m x k times k x n), split-BF16 tensor-core product. */
    public static native int gemm(long ctx, int m, int n, int k, double[] a, double[] b, double[] c);
    /** Complex FFT of interleaved (re, im) data; dir -1 forward, +1 inverse. */
    public static native int fft(long ctx, int n, int dir, double[] in, double[] out);
    /** Offload pattern of the Jacobi program: final p and residuals. */
    public static native int runPattern(long ctx, long gene, int hoist, int i, int j, int k, int iters,
                                        float omega, float[] p, double[] res);
    /** Serving: start, submit a GEMM (returns a ticket), wait (returns latency ms). */
    public static native int serveStart(long ctx, int slots, long budgetBytes, int queueCap);
    public static native long submitGemm(long ctx, int m, int n, int k, double[] a, double[] b, double[] c);
    public static native double await(long ctx, long ticket, int timeoutMs);
    public static native int serveStop(long ctx);
}
