/* NVTX injection library for the tracing test: records every range push and pop of the process
 * that loads it (through NVTX_INJECTION64_PATH) as lines "push <name>" / "pop" appended to the file
 * named by NVTX_RECORD_FILE. Host-only; needs the header-only NVTX v3 types. */
#include <stdio.h>
#include <stdlib.h>
#include <nvtx3/nvToolsExt.h>

static void record(const char *what, const char *name)
{
    const char *path = getenv("NVTX_RECORD_FILE");
    FILE *f = path ? fopen(path, "a") : NULL;
    if (!f) return;
    if (name) fprintf(f, "%s %s\n", what, name);
    else fprintf(f, "%s\n", what);
    fclose(f);
}

static int rec_push(const char *message)
{
    record("push", message);
    return 0;
}

static int rec_pop(void)
{
    record("pop", NULL);
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = NULL;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
    return 1;
}
