#define LPDEC_D 6
#include "lpdec_kclass.cuh"
