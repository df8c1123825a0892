/* A plain C99 program against include/ac.h and libacgb300.so: builds a
 * host-only automaton, saves it, loads it back, checks its statistics and
 * the refusal to scan a host-only automaton, and releases both (CPU only;
 * built and run by tests/test_abi_from_c.py). */
#include <stdio.h>
#include <string.h>
#include "ac.h"
int main(int argc, char **argv) {
    if (argc < 2) return 9;
    const char *p0 = "ACGT", *p1 = "GATTACA";
    const uint8_t *pats[2] = {(const uint8_t *)p0, (const uint8_t *)p1};
    uint32_t lens[2] = {4, 7};
    ac_build_opts o;
    memset(&o, 0, sizeof(o));
    o.alphabet = "ACGT";
    o.num_subsets = 1;
    o.device = -1;
    ac_automaton *a = NULL;
    if (ac_build(pats, lens, 2, &o, &a) != AC_OK) { printf("build: %s\n", ac_last_error()); return 1; }
    ac_stats_t st;
    if (ac_stats(a, &st) != AC_OK || st.num_patterns != 2) return 2;
    if (ac_save(a, argv[1]) != AC_OK) return 3;
    ac_automaton *b = NULL;
    if (ac_load(argv[1], -1, &b) != AC_OK) { printf("load: %s\n", ac_last_error()); return 4; }
    ac_stats_t sb;
    if (ac_stats(b, &sb) != AC_OK || sb.states != st.states) return 5;
    ac_result r;
    if (ac_scan(b, (const uint8_t *)"ACGT", 4, AC_U8, AC_HOST, NULL, &r) != AC_EINVAL) return 6;  /* host-only */
    printf("states %llu %s\n", (unsigned long long)sb.states, ac_strerror(AC_EINVAL));
    ac_free(a);
    ac_free(b);
    return 0;
}
