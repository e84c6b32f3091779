#define LPDEC_D 8
#include "lpdec_kclass.cuh"
