/*
 * opcount.cpp -- the oracle (hgks_oracle.c, unchanged) compiled as C++ with
 * every double replaced by the counting opc_double of opcount.hpp.  TEST
 * INFRASTRUCTURE ONLY.  The exported or_* entry points keep their C names and
 * their memory layout (opc_double is one double), so oracle/opcount.py calls
 * them with the same argument structures as the plain oracle; opc_reset and
 * opc_read clear and sum the per-thread operation counters.
 */
#include "opcount.hpp"

#ifdef _OPENMP
#include <omp.h>
#endif

unsigned long long opc_counts[256][8];

int opc_thread()
{
#ifdef _OPENMP
    return omp_get_thread_num() & 255;
#else
    return 0;
#endif
}

#define double opc_double
extern "C" {
#include "hgks_oracle.c"
}
#undef double

extern "C" void opc_reset(void) { memset(opc_counts, 0, sizeof opc_counts); }

extern "C" void opc_read(unsigned long long* out)
{
    for (int k = 0; k < OPC_KINDS; k++) {
        out[k] = 0;
        for (int t = 0; t < 256; t++) out[k] += opc_counts[t][k];
    }
}
