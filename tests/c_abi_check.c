/* A C99 caller of libhl.so: the header compiles as plain C, links, and the
 * argument checks that run before any CUDA call answer as include/hl.h states.
 * Needs no GPU.  Prints "ok" and exits 0, or names the first failed check. */
#include <stdio.h>
#include <string.h>

#include "hl.h"

#define CHECK(cond, what)                                       \
    do {                                                        \
        if (!(cond)) {                                          \
            printf("failed: %s (%s)\n", what, hl_last_error(0)); \
            return 1;                                           \
        }                                                       \
    } while (0)

int main(void)
{
    int64_t n1[1] = {8}, n2[2] = {8, 16};
    hl_solver *h = (hl_solver *)&n1;   /* must be overwritten with NULL on failure */
    CHECK(hl_create(4, 3, n1, 0.01, &h) == HL_EINVAL, "dim 4 rejected");
    CHECK(h == NULL, "no handle on failure");
    CHECK(strstr(hl_last_error(NULL), "dim") != NULL, "message names the argument");
    CHECK(hl_create(2, 7, n2, 0.01, &h) == HL_EINVAL, "m 7 rejected");
    CHECK(hl_create(2, 3, n2, 0.07, &h) == HL_EINVAL, "dt above min h rejected");
    CHECK(hl_create(1, 3, n1, 0.01, NULL) == HL_EINVAL, "NULL out rejected");
    CHECK(hl_step(NULL, 1) == HL_EINVAL, "hl_step on NULL");
    CHECK(hl_set_initial(NULL, NULL, NULL) == HL_EINVAL, "hl_set_initial on NULL");
    CHECK(hl_get_fields(NULL, NULL, NULL, NULL, NULL) == HL_EINVAL, "hl_get_fields on NULL");
    CHECK(hl_mlp_forward(NULL, NULL, 0, NULL) == HL_EINVAL, "hl_mlp_forward on NULL");
    CHECK(hl_mlp_last_error(NULL) != NULL, "mlp message never NULL");
    hl_destroy(NULL);
    hl_mlp_destroy(NULL);
    printf("ok\n");
    return 0;
}
