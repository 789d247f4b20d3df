/* Exhaustive check that the oracle's h1 is a bijection on 32-bit words:
 * every one of the 2^32 inputs maps to a distinct output.  Prints the number
 * of outputs hit (4294967296 for a bijection).  Links against liboracle. */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

uint32_t oracle_h1(uint32_t x);

static uint64_t* bits;
enum { NT = 16 };

static void* work(void* arg) {
    uint64_t t = (uint64_t)(uintptr_t)arg;
    uint64_t lo = (t << 32) / NT, hi = ((t + 1) << 32) / NT;
    for (uint64_t x = lo; x < hi; ++x) {
        uint32_t y = oracle_h1((uint32_t)x);
        __atomic_fetch_or(&bits[y >> 6], 1ull << (y & 63), __ATOMIC_RELAXED);
    }
    return NULL;
}

int main(void) {
    bits = (uint64_t*)calloc(1ull << 26, sizeof(uint64_t));
    if (!bits) return 2;
    pthread_t th[NT];
    for (uint64_t t = 0; t < NT; ++t) pthread_create(&th[t], NULL, work, (void*)(uintptr_t)t);
    for (int t = 0; t < NT; ++t) pthread_join(th[t], NULL);
    uint64_t hit = 0;
    for (uint64_t i = 0; i < (1ull << 26); ++i) hit += (uint64_t)__builtin_popcountll(bits[i]);
    printf("%llu\n", (unsigned long long)hit);
    return 0;
}
