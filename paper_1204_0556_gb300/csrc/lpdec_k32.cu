#define LPDEC_D 32
#include "lpdec_kclass.cuh"
