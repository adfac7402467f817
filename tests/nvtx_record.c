/* Test fixture: an NVTX injection library that appends every range push ("push <name>") and pop
 * ("pop") of the process to the file named by NVTX_RECORD_FILE.  Loaded by NVTX when the
 * environment variable NVTX_INJECTION64_PATH names it. */
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

static FILE* g_out;

static int rec_push(const char* name) {
  if (g_out) {
    fprintf(g_out, "push %s\n", name ? name : "");
    fflush(g_out);
  }
  return 0;
}
static int rec_pop(void) {
  if (g_out) {
    fputs("pop\n", g_out);
    fflush(g_out);
  }
  return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  const char* path = getenv("NVTX_RECORD_FILE");
  if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
  if (size <= NVTX_CBID_CORE_RangePop) return 0;
  g_out = fopen(path, "a");
  if (!g_out) return 0;
  *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
  *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
  return 1;
}
