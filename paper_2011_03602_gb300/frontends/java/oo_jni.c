/*
 * oo_jni.c -- JNI shim between OoNative.java and the C ABI (include/oo.h).
 * Arrays are pinned with Get/ReleasePrimitiveArrayCritical for synchronous
 * calls; for serving, the request's arrays are copied into C-heap buffers
 * that live until await() copies the result back (the JVM may move Java
 * arrays between calls).  Not built here: no JDK is installed.
 */
#include <jni.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oo.h"

typedef struct pending {
    uint64_t ticket;
    double *a, *b, *c;
    jdoubleArray out;
    size_t out_len;
    struct pending *next;
} pending;
static pending *g_pending = NULL;  /* guarded by the JVM monitor on OoNative.class */

static void throw_oo(JNIEnv *env, const char *what, oo_status s) {
    jclass ex = (*env)->FindClass(env, "java/lang/RuntimeException");
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, oo_status_str(s));
    (*env)->ThrowNew(env, ex, msg);
}

JNIEXPORT jlong JNICALL Java_oo_OoNative_create(JNIEnv *env, jclass cls, jint device) {
    (void)cls;
    oo_ctx *ctx = NULL;
    const oo_status s = oo_create(device, NULL, &ctx);
    if (s != OO_OK) throw_oo(env, "oo_create", s);
    return (jlong)(intptr_t)ctx;
}

JNIEXPORT void JNICALL Java_oo_OoNative_destroy(JNIEnv *env, jclass cls, jlong ctx) {
    (void)env;
    (void)cls;
    oo_destroy((oo_ctx *)(intptr_t)ctx);
}

JNIEXPORT jint JNICALL Java_oo_OoNative_lookupBlock(JNIEnv *env, jclass cls, jstring callee) {
    (void)cls;
    const char *name = (*env)->GetStringUTFChars(env, callee, NULL);
    int block = 0;
    const oo_status s = oo_lookup_block(name, OO_LANG_JAVA, &block);
    (*env)->ReleaseStringUTFChars(env, callee, name);
    return s == OO_OK ? block : 0;
}

JNIEXPORT jint JNICALL Java_oo_OoNative_gemm(JNIEnv *env, jclass cls, jlong ctx, jint m, jint n, jint k,
                                             jdoubleArray a, jdoubleArray b, jdoubleArray c) {
    (void)cls;
    double *pa = (*env)->GetPrimitiveArrayCritical(env, a, NULL);
    double *pb = (*env)->GetPrimitiveArrayCritical(env, b, NULL);
    double *pc = (*env)->GetPrimitiveArrayCritical(env, c, NULL);
    const oo_status s = oo_gemm_f64((oo_ctx *)(intptr_t)ctx, OO_PREC_SPLIT3_BF16, m, n, k, pa, k, pb, n, pc, n);
    (*env)->ReleasePrimitiveArrayCritical(env, c, pc, 0);
    (*env)->ReleasePrimitiveArrayCritical(env, b, pb, JNI_ABORT);
    (*env)->ReleasePrimitiveArrayCritical(env, a, pa, JNI_ABORT);
    return s;
}

JNIEXPORT jint JNICALL Java_oo_OoNative_fft(JNIEnv *env, jclass cls, jlong ctx, jint n, jint dir, jdoubleArray in,
                                            jdoubleArray out) {
    (void)cls;
    double *pi = (*env)->GetPrimitiveArrayCritical(env, in, NULL);
    double *po = (*env)->GetPrimitiveArrayCritical(env, out, NULL);
    const oo_status s = oo_fft_c128((oo_ctx *)(intptr_t)ctx, n, dir, pi, po);
    (*env)->ReleasePrimitiveArrayCritical(env, out, po, 0);
    (*env)->ReleasePrimitiveArrayCritical(env, in, pi, JNI_ABORT);
    return s;
}

JNIEXPORT jint JNICALL Java_oo_OoNative_runPattern(JNIEnv *env, jclass cls, jlong ctx, jlong gene, jint hoist,
                                                   jint i, jint j, jint k, jint iters, jfloat omega,
                                                   jfloatArray p, jdoubleArray res) {
    (void)cls;
    oo_jacobi prob = {i, j, k, iters, omega, 0};
    float *pp = (*env)->GetPrimitiveArrayCritical(env, p, NULL);
    double *pr = (*env)->GetPrimitiveArrayCritical(env, res, NULL);
    const oo_status s = oo_run_pattern((oo_ctx *)(intptr_t)ctx, (uint64_t)gene, hoist, &prob, pp, pr, NULL);
    (*env)->ReleasePrimitiveArrayCritical(env, res, pr, 0);
    (*env)->ReleasePrimitiveArrayCritical(env, p, pp, 0);
    return s;
}

JNIEXPORT jint JNICALL Java_oo_OoNative_serveStart(JNIEnv *env, jclass cls, jlong ctx, jint slots, jlong budget,
                                                   jint queue_cap) {
    (void)env;
    (void)cls;
    return oo_serve_start((oo_ctx *)(intptr_t)ctx, slots, (uint64_t)budget, queue_cap);
}

JNIEXPORT jlong JNICALL Java_oo_OoNative_submitGemm(JNIEnv *env, jclass cls, jlong ctx, jint m, jint n, jint k,
                                                    jdoubleArray a, jdoubleArray b, jdoubleArray c) {
    pending *q = calloc(1, sizeof(pending));
    q->a = malloc(sizeof(double) * (size_t)m * k);
    q->b = malloc(sizeof(double) * (size_t)k * n);
    q->c = malloc(sizeof(double) * (size_t)m * n);
    q->out_len = (size_t)m * n;
    (*env)->GetDoubleArrayRegion(env, a, 0, m * k, q->a);
    (*env)->GetDoubleArrayRegion(env, b, 0, k * n, q->b);
    q->out = (*env)->NewGlobalRef(env, c);
    oo_serve_req r;
    memset(&r, 0, sizeof r);
    r.kind = OO_BLOCK_GEMM;
    r.prec = OO_PREC_SPLIT3_BF16;
    r.m = m;
    r.n = n;
    r.k = k;
    r.client = OO_LANG_JAVA;
    r.in0 = q->a;
    r.in1 = q->b;
    r.out = q->c;
    const oo_status s = oo_submit((oo_ctx *)(intptr_t)ctx, &r, &q->ticket);
    if (s != OO_OK) {
        (*env)->DeleteGlobalRef(env, q->out);
        free(q->a);
        free(q->b);
        free(q->c);
        free(q);
        throw_oo(env, "oo_submit", s);
        return 0;
    }
    (*env)->MonitorEnter(env, cls);
    q->next = g_pending;
    g_pending = q;
    (*env)->MonitorExit(env, cls);
    return (jlong)q->ticket;
}

JNIEXPORT jdouble JNICALL Java_oo_OoNative_await(JNIEnv *env, jclass cls, jlong ctx, jlong ticket, jint timeout_ms) {
    double lat = -1.0;
    const oo_status s = oo_wait((oo_ctx *)(intptr_t)ctx, (uint64_t)ticket, timeout_ms, &lat);
    (*env)->MonitorEnter(env, cls);
    pending **pp = &g_pending, *q = NULL;
    while (*pp && (*pp)->ticket != (uint64_t)ticket) pp = &(*pp)->next;
    if (*pp && s != OO_ETIMEOUT) {
        q = *pp;
        *pp = q->next;
    }
    (*env)->MonitorExit(env, cls);
    if (q) {
        if (s == OO_OK) (*env)->SetDoubleArrayRegion(env, q->out, 0, (jsize)q->out_len, q->c);
        (*env)->DeleteGlobalRef(env, q->out);
        free(q->a);
        free(q->b);
        free(q->c);
        free(q);
    }
    if (s != OO_OK) throw_oo(env, "oo_wait", s);
    return lat;
}

JNIEXPORT jint JNICALL Java_oo_OoNative_serveStop(JNIEnv *env, jclass cls, jlong ctx) {
    (void)env;
    (void)cls;
    return oo_serve_stop((oo_ctx *)(intptr_t)ctx);
}
