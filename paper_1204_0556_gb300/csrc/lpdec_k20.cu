#define LPDEC_D 20
#include "lpdec_kclass.cuh"
