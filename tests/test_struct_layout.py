"""The binding's ctypes structures mirror include/aerafold.h field by field (CPU only): the
field names of every struct the header declares appear in the same order in the binding, and
the status-bit constants agree."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "aerafold.h")).read()


def header_fields(name):
    body = re.search(r"typedef struct " + name + r" \{(.*?)\} " + name + ";", HEADER, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[\w*\]", "", decl).strip()   # array fields: the name before [n]
        if not decl:
            continue
        # "int32_t n_zen;  double zen0_rad" style lines hold one declaration each after the split
        fields.append(re.findall(r"(\w+)\s*$", decl)[0])
    return fields


def test_structs_match_the_header():
    from paper_1507_07733_gb300 import binding
    for name in ("ar_config", "ar_pattern_desc", "ar_event", "ar_outputs", "ar_batch_limits", "ar_recon_out",
                 "ar_server_config", "ar_batch_plan_info"):
        cls = getattr(binding, name)
        assert [f[0] for f in cls._fields_] == header_fields(name), name


def test_status_bits_match_the_header():
    from paper_1507_07733_gb300 import binding
    for name in ("AR_STATUS_SINGULAR", "AR_STATUS_ZEN_CLAMP", "AR_STATUS_BAD_DIR", "AR_STATUS_BAD_PATTERN"):
        m = re.search(r"#define " + name + r" (\d+)u", HEADER)
        assert m and int(m.group(1)) == getattr(binding, name), name
